"""Train the learned-damping model (IPT_ACCEL_DAMPED) on the GPU.

    python -m paper_2012_14702_gb300.train_damping [--problems 40] [--epochs 40]

Training family (the edge of the Picard iteration's domain): n = 4096,
theta_i = i/4, symmetric Delta with N(0,1) * 0.04 * s entries, s ~ U[0.2, 1.5]
(seeds 100..); the model is evaluated on seeds from 1000.

Data: teacher rollouts.  From Z = E each step evaluates F(Z) and F(F(Z))
(``ipt_step_dense``, split-FP16 products), records the features of every
column (the solver's definition) and the secant damping
alpha* = -<D1, D2> / ||D2||^2 (D1 = F - Z, D2 = F(F(Z)) - 2 F + Z, clipped to
[0.05, 2]) as the target, and moves Z by the target damping.  Training: Adam on
the mean squared error of alpha, with the library's own model kernels
(``ipt_damping_grad`` / ``ipt_damping_adam``).  Writes the FP16 parameters to
MODEL_PATH.
"""

from __future__ import annotations

import argparse
import os
import time

import numpy as np
import torch

from paper_2012_14702_gb300 import ipt, workloads

EDGE_N, EDGE_THETA_STEP, EDGE_SCALE = 4096, 0.25, 0.04
MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "damping_model_fp16.npy")
N_PARAMS = ipt.DAMPING_PARAMS
EPS = 1e-30


def edge_problem(seed):
    """(M, theta, s) of the edge family for one seed."""
    s = float(workloads.rng(seed + 7919).uniform(0.2, 1.5))
    M, th = workloads.dense_symmetric(EDGE_N, EDGE_SCALE * s, seed, theta_step=EDGE_THETA_STEP)
    return M, th, s


def features(inc3, lam3):
    """The solver's six features per column from (3, k) histories (oldest first)."""
    i2, i1, i0 = inc3
    l2, l1, l0 = lam3
    e = EPS
    num, den = l0 - l1, l1 - l2
    q = torch.where(den != 0, num / torch.where(den != 0, den, torch.ones_like(den)),
                    torch.zeros_like(den)).clamp(-4.0, 4.0)
    return torch.stack([torch.log10(i0 + e), torch.log10((i0 + e) / (i1 + e)),
                        torch.log10((i1 + e) / (i2 + e)), q.float(),
                        torch.log10((den.abs() / (l1.abs() + e)).float() + e),
                        torch.log10((num.abs() / (l0.abs() + e)).float() + e)], dim=1)


def rollout(solver, M, th, max_steps=60, tol=1e-6):
    """Teacher rollout of one problem: lists of feature rows and targets."""
    Mg = torch.as_tensor(M, dtype=torch.float32, device="cuda")
    tg = torch.as_tensor(th, dtype=torch.float64, device="cuda")
    n = M.shape[0]
    Z = torch.eye(n, dtype=torch.float32, device="cuda")
    incs, lams, xs, ts = [], [], [], []
    for _ in range(max_steps):
        F, lam, norms = solver.step_dense(Mg, Z, theta=tg, precision="fp16x3")
        rho = norms["residual_abs"] / max(norms_r0(M, th), 1e-300)
        if not np.isfinite(rho) or rho > 1e6:
            break
        if rho <= tol:
            break
        D1 = F - Z
        incs.append((D1.double().norm(dim=0) / Z.double().norm(dim=0)).float())
        lams.append(lam.double())  # differences far below FP32 resolution of lam
        F2, _, _ = solver.step_dense(Mg, F, theta=tg, precision="fp16x3")
        D2 = (F2.double() - 2 * F.double() + Z.double())
        num = -(D1.double() * D2).sum(0)
        den = (D2 * D2).sum(0)
        target = torch.where(den > 0, num / torch.where(den > 0, den, torch.ones_like(den)),
                             torch.ones_like(den)).clamp(0.05, 2.0).float()
        if len(incs) >= 3:
            xs.append(features(torch.stack(incs[-3:]), torch.stack(lams[-3:])).float())
            ts.append(target)
            alpha = target
        else:
            alpha = torch.ones_like(target)
        Z = Z + alpha[None, :] * D1
    return xs, ts


_R0 = {}


def norms_r0(M, th):
    key = id(M)
    if key not in _R0:
        off = M - np.diag(np.diag(M))
        _R0[key] = float(np.linalg.norm(off))
    return _R0[key]


def train(X, T, epochs, batch, lr, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    p16 = torch.as_tensor(init_params(seed), device="cuda")
    master = p16.float().clone()
    grad = torch.zeros(N_PARAMS, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(grad)
    v = torch.zeros_like(grad)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    N = X.shape[0]
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(N, device="cuda", generator=g)
        loss.zero_()
        nb = 0
        for i in range(0, N, batch):
            idx = perm[i:i + batch]
            ipt.damping_grad(p16, X[idx].contiguous(), T[idx].contiguous(), grad, loss)
            step += 1
            ipt.damping_adam(master, p16, grad, m, v, lr, step)
            nb += 1
        print(f"epoch {ep}: mse {loss.item() / nb:.5f}", flush=True)
    return p16


def init_params(seed):
    """Uniform +-1/sqrt(fan_in) initial weights, FP16 (W1, b1, W2, b2, W3, b3)."""
    g = np.random.default_rng(seed)
    ni, nh = 6, 64
    parts = [g.uniform(-1, 1, (ni, nh)) / np.sqrt(ni), g.uniform(-1, 1, nh) / np.sqrt(ni),
             g.uniform(-1, 1, (nh, nh)) / np.sqrt(nh), g.uniform(-1, 1, nh) / np.sqrt(nh),
             g.uniform(-1, 1, (nh, 1)) / np.sqrt(nh), g.uniform(-1, 1, 1) / np.sqrt(nh)]
    return np.concatenate([x.reshape(-1) for x in parts]).astype(np.float16)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--problems", type=int, default=40)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--max-samples", type=int, default=2_000_000)
    ap.add_argument("--out", default=MODEL_PATH)
    a = ap.parse_args(argv)
    solver = ipt.Solver()
    xs, ts = [], []
    t0 = time.time()
    for p in range(a.problems):
        M, th, s = edge_problem(100 + p)
        x, t = rollout(solver, M, th)
        xs += x
        ts += t
        print(f"problem {p} (s = {s:.2f}): {len(x)} steps", flush=True)
    X = torch.cat(xs)
    T = torch.cat(ts)
    keep = torch.isfinite(X).all(1) & torch.isfinite(T)
    X, T = X[keep], T[keep]
    if X.shape[0] > a.max_samples:
        sel = torch.randperm(X.shape[0], device="cuda")[:a.max_samples]
        X, T = X[sel], T[sel]
    print(f"{X.shape[0]} samples in {time.time() - t0:.1f} s", flush=True)
    p16 = train(X, T, a.epochs, a.batch, a.lr, seed=1)
    np.save(a.out, p16.cpu().numpy())
    print(f"saved {a.out}", flush=True)


if __name__ == "__main__":
    main()
