"""GB300-native CRBM-aided Monte Carlo (arXiv:2008.05401): CRBM block-Gibbs
proposals with an exact Metropolis-Hastings correction for the 2D Ising model
and the Kitaev honeycomb model, as hand-written sm_103a CUDA behind a C ABI
(include/crbm.h).  This package holds the in-tree build and the thin binding.
"""
from .binding import (EXPORTS, FP64, ISING, KITAEV, MIXED, NOBS, Context, CrbmError, Graph, Job,  # noqa: F401
                      crbm_create, crbm_destroy, crbm_graph_create, crbm_graph_destroy, crbm_graph_launch,
                      crbm_init_chains, crbm_job_bytes, crbm_last_error,
                      crbm_load_model, crbm_read_energies, crbm_read_observables, crbm_read_state,
                      crbm_release, crbm_run, crbm_run_batch, crbm_sync, crbm_tune, crbm_write_state, load)
