"""Thin ctypes binding of libcrbm.so (declarations and contracts: include/crbm.h).

Argument marshalling only: every step of the sampler runs in the CUDA
library.  The module-level ``crbm_*`` functions mirror the C entry points one
to one; ``Context`` / ``Job`` wrap them with torch tensors for device memory
and numpy arrays for host data.  Loading fails loudly when the library has
not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

ISING, KITAEV = 0, 1
FP64, MIXED = 0, 1
NOBS = 4
STATUS = {0: "CRBM_OK", -1: "CRBM_EINVAL", -2: "CRBM_ENOMEM", -3: "CRBM_ECUDA", -4: "CRBM_ETIMEOUT",
          -5: "CRBM_EBUSY"}

_lib = None


class CrbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class TrainProblem(C.Structure):
    """crbm_train_problem (include/crbm.h): device pointers and sizes of one training problem."""
    _fields_ = [("K", C.c_int), ("k", C.c_int), ("L", C.c_int), ("n_samples", C.c_int),
                ("samples", C.c_void_p), ("targets", C.c_void_p), ("order", C.c_void_p),
                ("theta", C.c_void_p), ("adam_m", C.c_void_p), ("adam_v", C.c_void_p),
                ("adam_t", C.c_void_p), ("losses", C.c_void_p)]


_SIGS = {
    "crbm_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_size_t]),
    "crbm_destroy": (C.c_int, [C.c_void_p]),
    "crbm_last_error": (C.c_char_p, [C.c_void_p]),
    "crbm_load_model": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_double,
                                  C.c_void_p, C.POINTER(C.c_int)]),
    "crbm_load_lcrbm": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_double,
                                  C.c_void_p, C.POINTER(C.c_int)]),
    "crbm_job_bytes": (C.c_size_t, [C.c_int, C.c_int, C.c_int, C.c_int]),
    "crbm_init_chains": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                   C.c_uint64, C.c_uint64, C.c_int, C.c_void_p, C.c_void_p, C.c_size_t,
                                   C.POINTER(C.c_int)]),
    "crbm_run": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "crbm_run_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int,
                                 C.c_void_p]),
    "crbm_graph_create": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int,
                                    C.c_int, C.POINTER(C.c_int)]),
    "crbm_graph_launch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "crbm_graph_destroy": (C.c_int, [C.c_void_p, C.c_int]),
    "crbm_pt_run": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_int, C.c_int, C.c_void_p]),
    "crbm_local_run": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_int, C.c_int, C.c_void_p]),
    "crbm_set_trace": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64]),
    "crbm_autocorr": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_void_p,
                                C.c_void_p, C.c_void_p]),
    "crbm_autocorr_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_void_p,
                                        C.c_void_p, C.c_void_p]),
    "crbm_train_epochs": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_double, C.c_double,
                                    C.c_double, C.c_double, C.c_void_p]),
    "crbm_update_model": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_double, C.c_void_p]),
    "crbm_probe_peaks": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "crbm_tune": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "crbm_sync": (C.c_int, [C.c_void_p, C.c_int]),
    "crbm_set_wait_limit": (C.c_int, [C.c_void_p, C.c_int64]),
    "crbm_probe_wait": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_void_p]),
    "crbm_set_tensor_cores": (C.c_int, [C.c_void_p, C.c_int]),
    "crbm_read_energies": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "crbm_read_observables": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "crbm_read_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_uint64)]),
    "crbm_write_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_uint64, C.c_int]),
    "crbm_write_states": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "crbm_read_states": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "crbm_release": (C.c_int, [C.c_void_p, C.c_int]),
}
EXPORTS = tuple(_SIGS)


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libcrbm.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first (__graft_entry__.build())")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(ctx, rc):
    if rc != 0:
        msg = load().crbm_last_error(ctx).decode() if ctx else ""
        raise CrbmError(rc, msg)


# ---- one-to-one wrappers of the C entry points --------------------------------
def crbm_create(device: int = 0, hbm_budget_bytes: int = 0):
    h = C.c_void_p()
    _check(None, load().crbm_create(C.byref(h), device, hbm_budget_bytes))
    return h


def crbm_destroy(ctx):
    _check(None, load().crbm_destroy(ctx))


def crbm_last_error(ctx) -> str:
    return load().crbm_last_error(ctx).decode()


def crbm_load_model(ctx, kind, W, v_bias, h_bias) -> int:
    W = np.ascontiguousarray(W, dtype=np.float64)
    hb = np.ascontiguousarray(h_bias, dtype=np.float64)
    K, k, _ = W.shape
    mid = C.c_int()
    _check(ctx, load().crbm_load_model(ctx, kind, K, k, _ptr(W), float(v_bias), _ptr(hb), C.byref(mid)))
    return mid.value


def crbm_load_lcrbm(ctx, kind, W, v_bias, h_bias) -> int:
    """W: (2 edge + 1, K, k, k) class kernels (left edge, right edge, bulk)."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    hb = np.ascontiguousarray(h_bias, dtype=np.float64)
    ncls, K, k, _ = W.shape
    mid = C.c_int()
    _check(ctx, load().crbm_load_lcrbm(ctx, kind, K, k, (ncls - 1) // 2, _ptr(W), float(v_bias), _ptr(hb),
                                       C.byref(mid)))
    return mid.value


def crbm_job_bytes(kind, L, n_chains, precision=FP64) -> int:
    return int(load().crbm_job_bytes(kind, L, n_chains, precision))


def crbm_init_chains(ctx, model_id, L, T, J, seed, chain_id_base, init_bits, dev_ptr, dev_bytes) -> int:
    T = np.ascontiguousarray(T, dtype=np.float64)
    J = np.ascontiguousarray(J, dtype=np.float64)
    bits = None if init_bits is None else np.ascontiguousarray(init_bits, dtype=np.uint32)
    jid = C.c_int()
    _check(ctx, load().crbm_init_chains(ctx, model_id, L, len(T), _ptr(T), _ptr(J), seed, chain_id_base,
                                        0 if bits is None else 1, _ptr(bits), C.c_void_p(dev_ptr),
                                        dev_bytes, C.byref(jid)))
    return jid.value


def crbm_run(ctx, job_id, S, g=1, correct=1, precision=FP64, stream=0):
    _check(ctx, load().crbm_run(ctx, job_id, S, g, correct, precision, C.c_void_p(stream)))


def crbm_run_batch(ctx, job_ids, S, g=1, correct=1, precision=FP64, stream=0):
    ids = np.ascontiguousarray(job_ids, dtype=np.int32)
    _check(ctx, load().crbm_run_batch(ctx, len(ids), _ptr(ids), S, g, correct, precision, C.c_void_p(stream)))


def crbm_graph_create(ctx, job_ids, S, g=1, correct=1, precision=FP64, repeats=1) -> int:
    ids = np.ascontiguousarray(job_ids, dtype=np.int32)
    gid = C.c_int()
    _check(ctx, load().crbm_graph_create(ctx, len(ids), _ptr(ids), S, g, correct, precision, repeats,
                                         C.byref(gid)))
    return gid.value


def crbm_graph_launch(ctx, graph_id, stream=0):
    _check(ctx, load().crbm_graph_launch(ctx, graph_id, C.c_void_p(stream)))


def crbm_graph_destroy(ctx, graph_id):
    _check(ctx, load().crbm_graph_destroy(ctx, graph_id))


def crbm_pt_run(ctx, phys_job, rbm_job, cycles, g=1, precision=FP64, stream=0):
    _check(ctx, load().crbm_pt_run(ctx, phys_job, rbm_job, cycles, g, precision, C.c_void_p(stream)))


def crbm_local_run(ctx, job_id, sweeps, exchange=0, precision=FP64, stream=0):
    _check(ctx, load().crbm_local_run(ctx, job_id, sweeps, exchange, precision, C.c_void_p(stream)))


def crbm_set_trace(ctx, job_id, dev_ptr, capacity_steps):
    _check(ctx, load().crbm_set_trace(ctx, job_id, C.c_void_p(dev_ptr), capacity_steps))


def crbm_autocorr(ctx, dev_ptr, n_series, length, c=5.0, stream=0):
    tau = np.empty(n_series)
    win = np.empty(n_series, dtype=np.int64)
    _check(ctx, load().crbm_autocorr(ctx, C.c_void_p(dev_ptr), n_series, length, c, _ptr(tau), _ptr(win),
                                     C.c_void_p(stream)))
    return tau, win


def crbm_autocorr_noalloc(ctx, dev_ptr, n_series, length, c=5.0, stream=0):
    tau = np.empty(n_series)
    win = np.empty(n_series, dtype=np.int64)
    _check(ctx, load().crbm_autocorr_noalloc(ctx, C.c_void_p(dev_ptr), n_series, length, c, _ptr(tau),
                                             _ptr(win), C.c_void_p(stream)))
    return tau, win


def crbm_train_epochs(ctx, problems, batch=20, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, stream=0):
    arr = (TrainProblem * max(len(problems), 1))(*problems)
    _check(ctx, load().crbm_train_epochs(ctx, len(problems), C.cast(arr, C.c_void_p), batch, lr, b1, b2, eps,
                                         C.c_void_p(stream)))


def crbm_update_model(ctx, model_id, W, v_bias, h_bias):
    W = np.ascontiguousarray(W, dtype=np.float64)
    hb = np.ascontiguousarray(h_bias, dtype=np.float64)
    _check(ctx, load().crbm_update_model(ctx, model_id, _ptr(W), float(v_bias), _ptr(hb)))


def crbm_probe_peaks(ctx):
    """Measured (FP32, FP64) FMA throughput of the context's device, TFLOP/s."""
    a, b = C.c_double(), C.c_double()
    _check(ctx, load().crbm_probe_peaks(ctx, C.byref(a), C.byref(b)))
    return a.value, b.value


def crbm_tune(ctx, model_id, L, precision=FP64):
    nc, us = C.c_int(), C.c_double()
    _check(ctx, load().crbm_tune(ctx, model_id, L, precision, C.byref(nc), C.byref(us)))
    return nc.value, us.value


def crbm_sync(ctx, job_id):
    _check(ctx, load().crbm_sync(ctx, job_id))


def crbm_set_wait_limit(ctx, cycles):
    _check(ctx, load().crbm_set_wait_limit(ctx, int(cycles)))


def crbm_probe_wait(ctx, limit_cycles, arrive, stream=0):
    _check(ctx, load().crbm_probe_wait(ctx, int(limit_cycles), int(arrive), C.c_void_p(stream)))


def crbm_set_tensor_cores(ctx, enable):
    _check(ctx, load().crbm_set_tensor_cores(ctx, int(enable)))


def crbm_read_energies(ctx, job_id, n):
    lp, F, E = (np.empty(n) for _ in range(3))
    _check(ctx, load().crbm_read_energies(ctx, job_id, _ptr(lp), _ptr(F), _ptr(E)))
    return lp, F, E


def crbm_read_observables(ctx, job_id, n):
    sums = np.empty((n, NOBS))
    acc = np.empty(n, dtype=np.int64)
    rec = np.empty((n, 2), dtype=np.int64)
    _check(ctx, load().crbm_read_observables(ctx, job_id, _ptr(sums), _ptr(acc), _ptr(rec)))
    return sums, acc, rec


def crbm_read_state(ctx, job_id, n, L, out=None):
    """Lattices (into `out`, e.g. a pinned buffer, when given) and step counter."""
    bits = np.empty((n, (L * L + 31) // 32), dtype=np.uint32) if out is None else out
    if bits.dtype != np.uint32 or bits.shape != (n, (L * L + 31) // 32) or not bits.flags.c_contiguous:
        raise ValueError("out must be a C-contiguous uint32 array of shape (n, ceil(L*L/32))")
    step = C.c_uint64()
    _check(ctx, load().crbm_read_state(ctx, job_id, _ptr(bits), C.byref(step)))
    return bits, step.value


def crbm_write_state(ctx, job_id, bits, step, precision=FP64):
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    _check(ctx, load().crbm_write_state(ctx, job_id, _ptr(bits), step, precision))


def crbm_write_states(ctx, job_ids, bits_list, steps, precision=FP64):
    """crbm_write_state for several jobs, one evaluation launch for all."""
    n = len(job_ids)
    arrs = [np.ascontiguousarray(b, dtype=np.uint32) for b in bits_list]
    ids = (C.c_int * n)(*job_ids)
    ptrs = (C.c_void_p * n)(*[a.ctypes.data for a in arrs])
    st = (C.c_uint64 * n)(*steps)
    _check(ctx, load().crbm_write_states(ctx, n, ids, ptrs, st, precision))


def crbm_read_states(ctx, job_ids, bits_out, sums_out):
    """Lattices into bits_out[i] and observable sums into sums_out[i] (C-contiguous
    uint32 / float64 arrays of the jobs' shapes, or None) for several jobs,
    one synchronisation; returns the step counters."""
    n = len(job_ids)
    for b in bits_out:
        if b is not None and (b.dtype != np.uint32 or not b.flags.c_contiguous):
            raise ValueError("bits_out entries must be C-contiguous uint32 arrays")
    for x in sums_out:
        if x is not None and (x.dtype != np.float64 or not x.flags.c_contiguous):
            raise ValueError("sums_out entries must be C-contiguous float64 arrays")
    ids = (C.c_int * n)(*job_ids)
    bp = (C.c_void_p * n)(*[None if b is None else b.ctypes.data for b in bits_out])
    sp = (C.c_void_p * n)(*[None if x is None else x.ctypes.data for x in sums_out])
    st = (C.c_uint64 * n)()
    _check(ctx, load().crbm_read_states(ctx, n, ids, bp, st, sp))
    return [int(v) for v in st]


def crbm_release(ctx, job_id):
    _check(ctx, load().crbm_release(ctx, job_id))


# ---- convenience layer: torch tensors hold the job memory ---------------------
class Job:
    def __init__(self, ctx: "Context", job_id: int, L: int, n: int, mem):
        self.ctx, self.id, self.L, self.n, self.mem = ctx, job_id, L, n, mem
        self.step = 0

    def run(self, S, g=1, correct=True, precision=FP64, stream=None):
        crbm_run(self.ctx.h, self.id, S, g, int(correct), precision, _stream_handle(stream))
        self.step += S
        return self

    def sync(self):
        crbm_sync(self.ctx.h, self.id)

    def energies(self):
        return crbm_read_energies(self.ctx.h, self.id, self.n)

    def observables(self):
        return crbm_read_observables(self.ctx.h, self.id, self.n)

    def state(self, out=None):
        return crbm_read_state(self.ctx.h, self.id, self.n, self.L, out)

    def write_state(self, bits, step, precision=FP64):
        crbm_write_state(self.ctx.h, self.id, bits, step, precision)
        self.step = step

    def local_run(self, sweeps, exchange=False, precision=FP64, stream=None):
        """Local-update Metropolis sweeps (optionally with temperature exchange)."""
        crbm_local_run(self.ctx.h, self.id, sweeps, int(exchange), precision, _stream_handle(stream))
        self.step += sweeps
        return self

    def set_trace(self, steps):
        """Record E_phys of every chain for the next `steps` steps; returns the
        (steps, n) float64 torch tensor that receives it (None: stop)."""
        import torch
        if steps is None:
            crbm_set_trace(self.ctx.h, self.id, 0, 0)
            self.trace = None
            return None
        self.trace = torch.full((steps, self.n), float("nan"), dtype=torch.float64,
                                device=f"cuda:{self.ctx.device}")
        crbm_set_trace(self.ctx.h, self.id, self.trace.data_ptr(), steps)
        return self.trace

    def release(self):
        crbm_release(self.ctx.h, self.id)
        self.mem = None


class Graph:
    def __init__(self, ctx: "Context", gid: int, jobs, steps: int):
        self.ctx, self.id, self.jobs, self.steps = ctx, gid, list(jobs), steps

    def launch(self, stream=None):
        crbm_graph_launch(self.ctx.h, self.id, _stream_handle(stream))
        for j in self.jobs:
            j.step += self.steps

    def destroy(self):
        crbm_graph_destroy(self.ctx.h, self.id)


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Context:
    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.device = device
        self.h = crbm_create(device, hbm_budget_bytes)

    def close(self):
        if self.h:
            crbm_destroy(self.h)
            self.h = None

    def load_model(self, kind, W, v_bias, h_bias) -> int:
        return crbm_load_model(self.h, kind, W, v_bias, h_bias)

    def load_lcrbm(self, kind, W, v_bias, h_bias) -> int:
        """Locally connected CRBM for the open-boundary Kitaev model; W (2 edge + 1, K, k, k)."""
        return crbm_load_lcrbm(self.h, kind, W, v_bias, h_bias)

    def new_job(self, model_id, kind, L, T, J, seed, chain_id_base=0, init_bits=None, precision=FP64,
                mem=None) -> Job:
        import torch
        T = np.atleast_1d(np.asarray(T, dtype=np.float64))
        nbytes = crbm_job_bytes(kind, L, len(T), precision)
        if mem is None:
            mem = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=f"cuda:{self.device}")
        jid = crbm_init_chains(self.h, model_id, L, T, J, seed, chain_id_base, init_bits,
                               mem.data_ptr() if len(T) else 0, mem.numel())
        return Job(self, jid, L, len(T), mem)

    def update_model(self, model_id, W, v_bias, h_bias):
        """New parameters for an existing model (same K, k)."""
        crbm_update_model(self.h, model_id, W, v_bias, h_bias)

    def set_tensor_cores(self, enable: bool):
        """Run later proposals of eligible jobs (Ising, mixed, L = 128, 64, 32 or 16, K <= 4,
        k <= 5) on the tensor-core kernel (True, default) or the table kernel."""
        crbm_set_tensor_cores(self.h, enable)

    def tune(self, model_id, L, precision=FP64):
        """Pick the fastest chains-per-CTA for (model, L); returns (nc, us per chain-proposal)."""
        return crbm_tune(self.h, model_id, L, precision)

    def graph(self, jobs, S, g=1, correct=True, precision=FP64, repeats=1) -> "Graph":
        """Capture `repeats` batched runs of S proposals into a replayable CUDA graph."""
        gid = crbm_graph_create(self.h, [j.id for j in jobs], S, g, int(correct), precision, repeats)
        return Graph(self, gid, jobs, S * repeats)

    def pt_run(self, phys: Job, rbm: Job, cycles, g=1, precision=FP64, stream=None):
        """Parallel-tempering exchange correction: `cycles` cycles of RBM
        proposals, physical <-> RBM swaps and neighbour temperature exchanges."""
        crbm_pt_run(self.h, phys.id, rbm.id, cycles, g, precision, _stream_handle(stream))
        phys.step += cycles
        rbm.step += cycles

    def autocorr(self, series, c=5.0, stream=None):
        """tau_int and window of every column of a (length, n) float64 CUDA tensor."""
        series = series.contiguous()
        return crbm_autocorr(self.h, series.data_ptr(), series.shape[1], series.shape[0], c,
                             _stream_handle(stream))

    def write_states(self, jobs, bits_list, steps, precision=FP64):
        """Job.write_state for several jobs of this context, one evaluation launch."""
        crbm_write_states(self.h, [j.id for j in jobs], bits_list, steps, precision)
        for j, st in zip(jobs, steps):
            j.step = st

    def read_states(self, jobs, bits_out, sums_out):
        """Lattices and observable sums of several jobs into the given arrays
        (shapes (n, ceil(L*L/32)) uint32 and (n, NOBS) float64; None skips),
        one synchronisation; returns the step counters."""
        for j, b, x in zip(jobs, bits_out, sums_out):
            if b is not None and b.shape != (j.n, (j.L * j.L + 31) // 32):
                raise ValueError("bits_out shape")
            if x is not None and x.shape != (j.n, NOBS):
                raise ValueError("sums_out shape")
        return crbm_read_states(self.h, [j.id for j in jobs], bits_out, sums_out)

    def run_batch(self, jobs, S, g=1, correct=True, precision=FP64, stream=None):
        crbm_run_batch(self.h, [j.id for j in jobs], S, g, int(correct), precision, _stream_handle(stream))
        for j in jobs:
            j.step += S
