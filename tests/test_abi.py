"""The C-ABI library builds, loads and exports every entry point include/crbm.h
declares (CPU only: no compute call needs a GPU here)."""
import ctypes
import os
import re

import pytest

from _common import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "crbm.h")).read()
    return sorted(set(re.findall(r"CRBM_API\s+[\w\s\*]+?\b(crbm_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("crbm_create", "crbm_load_model", "crbm_init_chains", "crbm_run", "crbm_run_batch",
              "crbm_sync", "crbm_read_energies", "crbm_read_observables", "crbm_read_state",
              "crbm_write_state", "crbm_release", "crbm_job_bytes", "crbm_last_error", "crbm_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2008_05401_gb300 import binding
    lib = ctypes.CDLL(binding.lib_path())
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(binding.EXPORTS) == set(_declared())


def test_host_only_calls_without_gpu():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2008_05401_gb300 import binding
    # sizes are pure host arithmetic
    b = binding.crbm_job_bytes(0, 128, 4096, 1)
    assert b >= 4096 * 512 * 4 and b % 256 == 0
    assert binding.crbm_job_bytes(0, 100, 4, 0) == 0          # L=100 unsupported for Ising
    assert binding.crbm_job_bytes(1, 13, 4, 0) == 0           # Kitaev L <= 12
    assert binding.crbm_job_bytes(0, 16, 0, 0) == 0           # empty job
    # Kitaev jobs also hold the spectrum of every lattice (L*L FP64 values)
    assert binding.crbm_job_bytes(1, 12, 10, 0) >= binding.crbm_job_bytes(0, 12, 10, 0) + 10 * 144 * 8
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        with pytest.raises(binding.CrbmError):
            binding.crbm_create(0)
