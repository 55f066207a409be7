"""The paper's CRBM trainer (Sec. II, App. A, Algorithm 1) driven from the host.

Every arithmetic step runs in the CUDA library: the epochs of minibatch ADAM
steps (``crbm_train_epochs``, one CTA per problem), the physical samples
(local-update Metropolis sweeps, ``crbm_local_run``), the buffer of RBM
samples (uncorrected Gibbs proposals, ``crbm_run`` with correct = 0) and their
targets (FP64 log pi of the job).  This module only moves lattices, targets
and parameters between jobs and the trainer's device tensors.

Parameters are the flat FP64 vector [W (K*k*k), v_bias, h_bias (K)] of
Algorithm 1.  Targets are t = -log pi (beta E for the Ising model).  Many
problems (one CRBM per temperature, as in Sec. IV) train side by side: each
epoch of all of them is one kernel launch.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import binding as B


@dataclass
class Problem:
    """Device state of one training problem (torch tensors on the context's device)."""
    K: int
    k: int
    L: int
    theta: object
    m: object
    v: object
    t: object

    @classmethod
    def new(cls, ctx: B.Context, K, k, L, theta0):
        import torch
        dev = f"cuda:{ctx.device}"
        th = torch.tensor(np.asarray(theta0, dtype=np.float64), device=dev)
        return cls(K, k, L, th, torch.zeros_like(th), torch.zeros_like(th),
                   torch.zeros(1, dtype=torch.int64, device=dev))

    def params(self):
        """(W (K, k, k), h_bias (K,), v_bias) on the host."""
        th = self.theta.cpu().numpy()
        n = self.K * self.k * self.k
        return th[:n].reshape(self.K, self.k, self.k), th[n + 1:].copy(), float(th[n])


def train_epochs(ctx: B.Context, problems, samples, targets, orders, batch=20, lr=1e-3, b1=0.9, b2=0.999,
                 eps=1e-8, stream=None):
    """One epoch of every problem in one launch.  samples[i]: (n_i, words)
    uint32 device tensor of packed lattices, targets[i]: (n_i,) float64,
    orders[i]: (n_i,) int32.  Returns the per-minibatch loss tensors."""
    import torch
    descs, losses = [], []
    for pr, x, t, o in zip(problems, samples, targets, orders):
        n = int(t.shape[0])
        ls = torch.empty(max(1, (n + batch - 1) // batch), dtype=torch.float64, device=t.device)
        losses.append(ls)
        descs.append(B.TrainProblem(pr.K, pr.k, pr.L, n, x.data_ptr(), t.data_ptr(), o.data_ptr(),
                                    pr.theta.data_ptr(), pr.m.data_ptr(), pr.v.data_ptr(), pr.t.data_ptr(),
                                    ls.data_ptr()))
    B.crbm_train_epochs(ctx.h, descs, batch, lr, b1, b2, eps, B._stream_handle(stream))
    return losses


def pretrain(ctx: B.Context, kind, L, Ts, J, K, k, theta0, n_random, seed, max_epochs, order_fn, M=20, patience=1,
             rel_tol=1e-4, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """Pre-training on random states (App. A; Sec. IV; App. D) for every
    temperature of Ts side by side.

    n_random uniform lattices, drawn on the device from the init tag of chains
    0 .. n_random-1 of `seed`, serve every temperature; their targets
    t = -log pi at each temperature come from one FP64 evaluation per
    temperature.  Each epoch of all problems still training is one launch
    (visiting order order_fn(n_random, epoch)); a problem stops once for
    `patience` epochs its epoch loss (the mean of its minibatch losses) has
    not fallen below (1 - rel_tol) times the loss of its last epoch that did,
    or after max_epochs, and keeps the parameters of its lowest-loss epoch.  Returns
    (problems, per-problem lists of epoch losses)."""
    import torch
    dev = f"cuda:{ctx.device}"
    zero = ctx.load_model(kind, np.zeros((K, k, k)), 0.0, np.zeros(K))
    x = ctx.new_job(zero, kind, L, np.full(n_random, Ts[0]), J, seed, 0, None, B.FP64)
    bits, _ = x.state()
    x.release()
    xs = torch.tensor(bits.view(np.int32), device=dev)
    ts = []
    for T in Ts:
        job = ctx.new_job(zero, kind, L, np.full(n_random, T), J, seed, 0, bits, B.FP64)
        lp, _, _ = job.energies()
        job.release()
        ts.append(torch.tensor(-lp, device=dev))
    probs = [Problem.new(ctx, K, k, L, theta0) for _ in Ts]
    best = [np.inf] * len(Ts)                 # lowest epoch loss and its parameters
    best_theta = [pr.theta.clone() for pr in probs]
    level = [np.inf] * len(Ts)                # loss at the last decrease by more than rel_tol
    stale = [0] * len(Ts)
    active = [True] * len(Ts)
    history = [[] for _ in Ts]
    for e in range(max_epochs):
        act = [i for i in range(len(Ts)) if active[i]]
        if not act:
            break
        order = torch.tensor(np.asarray(order_fn(n_random, e), dtype=np.int32), device=dev)
        losses = train_epochs(ctx, [probs[i] for i in act], [xs] * len(act), [ts[i] for i in act],
                              [order] * len(act), M, lr, b1, b2, eps)
        for i, ls in zip(act, losses):
            loss = float(ls.mean())
            history[i].append(loss)
            if loss < best[i]:
                best[i] = loss
                best_theta[i] = probs[i].theta.clone()
            if loss < level[i] * (1.0 - rel_tol):
                level[i], stale[i] = loss, 0
            else:
                stale[i] += 1
                active[i] = stale[i] < patience
    for pr, th in zip(probs, best_theta):
        pr.theta.copy_(th)
    return probs, history


def algorithm1(ctx: B.Context, kind, L, Ts, J, K, k, theta0, n_phys, phys_sweeps, phys_seed, n_train, ub, g,
               rbm_seed, epochs, order_fn, M=20, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, pre=None):
    """Algorithm 1 for every temperature of Ts side by side.

    Physical samples: the final lattices of n_phys local-Metropolis chains
    (seed phys_seed, chain ids 0..n_phys-1) after phys_sweeps sweeps from
    random lattices.  RBM buffer: ub chains (seed rbm_seed, ids 0..ub-1) from
    random lattices; each refresh is one uncorrected proposal of g Gibbs steps
    with the current parameters, its lattices put in front of the buffer,
    which is cut to n_train.  Each epoch: refresh, then one epoch over buffer
    + physical samples in the order order_fn(n, epoch).  theta0 gives the
    initial parameters of every problem; pre (keyword arguments of
    ``pretrain``: n_random, seed, max_epochs, order_fn and optionally
    patience, rel_tol) runs the pre-training step first, and each
    temperature's main loop starts from its pre-trained parameters with a
    fresh ADAM state.  Returns (problems, mean loss per epoch and
    temperature)."""
    import torch
    dev = f"cuda:{ctx.device}"
    theta0s = [theta0] * len(Ts)
    if pre is not None:
        pp, _ = pretrain(ctx, kind, L, Ts, J, K, k, theta0, M=M, lr=lr, b1=b1, b2=b2, eps=eps, **pre)
        theta0s = [pr.theta.cpu().numpy() for pr in pp]
    zero = ctx.load_model(kind, np.zeros((K, k, k)), 0.0, np.zeros(K))
    probs, phys_bits, phys_t, bufs, rings = [], [], [], [], []
    for T, th0 in zip(Ts, theta0s):
        x = ctx.new_job(zero, kind, L, np.full(n_phys, T), J, phys_seed, 0, None, B.FP64)
        x.local_run(phys_sweeps)
        bits, _ = x.state()
        lp, _, _ = x.energies()
        phys_bits.append(bits)
        phys_t.append(-lp)
        x.release()
        pr = Problem.new(ctx, K, k, L, th0)
        probs.append(pr)
        W, hb, vb = pr.params()
        mid = ctx.load_model(kind, W, vb, hb)
        bufs.append((mid, ctx.new_job(mid, kind, L, np.full(ub, T), J, rbm_seed, 0, None, B.FP64)))
        rings.append((np.zeros((0, bits.shape[1]), dtype=np.uint32), np.zeros(0)))

    def refresh(i):
        pr, (mid, job) = probs[i], bufs[i]
        W, hb, vb = pr.params()
        ctx.update_model(mid, W, vb, hb)
        job.run(1, g=g, correct=False, precision=B.FP64)
        bits, _ = job.state()
        lp, _, _ = job.energies()
        rb, rt = rings[i]
        rings[i] = (np.concatenate([bits, rb])[:n_train], np.concatenate([-lp, rt])[:n_train])

    for i in range(len(Ts)):
        while len(rings[i][1]) < n_train:
            refresh(i)
    history = []
    for e in range(epochs):
        xs, ts, os_ = [], [], []
        for i in range(len(Ts)):
            refresh(i)
            rb, rt = rings[i]
            xb = np.concatenate([rb, phys_bits[i]])
            tt = np.concatenate([rt, phys_t[i]])
            xs.append(torch.tensor(xb.view(np.int32), device=dev))
            ts.append(torch.tensor(tt, device=dev))
            os_.append(torch.tensor(np.asarray(order_fn(len(tt), e), dtype=np.int32), device=dev))
        losses = train_epochs(ctx, probs, xs, ts, os_, M, lr, b1, b2, eps)
        history.append([float(ls.mean()) for ls in losses])
    for _, job in bufs:
        job.release()
    return probs, np.array(history)
