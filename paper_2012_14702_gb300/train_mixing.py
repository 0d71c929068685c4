"""Train the learned damping-and-mixing model (IPT_ACCEL_MIXING) on the GPU.

    python -m paper_2012_14702_gb300.train_mixing [--problems 40] [--epochs 40]

Training family: the learned-damping one (train_damping: n = 4096,
theta_i = i/4, symmetric Delta N(0,1) * 0.04 * s, s ~ U[0.2, 1.5], seeds 100..).

Data: teacher rollouts.  From Z = E each step evaluates F(Z) (``ipt_step_dense``,
split-FP16 products) and, once a previous pair is known, two more points: the
Anderson point y_a + r_a (gamma = gamma_ls) and the Picard point F(Z).  Per column
the target gamma* is the candidate with the smaller residual there, and alpha*
the secant damping of that candidate's step (the oracle's statement:
oracle/mixing.py targets).  Features are the solver's seven.  The rollout follows
the target step from the fourth evaluation on.  Training: Adam on the mean squared
error of (alpha, gamma) with the library's own model kernels (``ipt_mixing_grad`` /
``ipt_mixing_adam``).  Writes the FP16 parameters to MODEL_PATH.
"""

from __future__ import annotations

import argparse
import os
import time

import numpy as np
import torch

from paper_2012_14702_gb300 import ipt
from paper_2012_14702_gb300.train_damping import (EDGE_N, EDGE_SCALE, EDGE_THETA_STEP,
                                                  edge_problem, norms_r0)
from paper_2012_14702_gb300.train_damping import features as damping_features

MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mixing_model_fp16.npy")
N_PARAMS = ipt.MIXING_PARAMS
GAMMA_CLIP = 1.9

__all__ = ["EDGE_N", "EDGE_SCALE", "EDGE_THETA_STEP", "MODEL_PATH", "main"]


def gamma_ls(f, fp):
    """<f - fp, f> / ||f - fp||^2 per column (0 where the difference vanishes)."""
    df = (f - fp).double()
    num = (df * f.double()).sum(0)
    den = (df * df).sum(0)
    return torch.where(den > 0, num / torch.where(den > 0, den, torch.ones_like(den)),
                       torch.zeros_like(den))


def rollout(solver, M, th, max_steps=60, tol=1e-6):
    """Teacher rollout of one problem: lists of feature rows and (alpha, gamma) targets."""
    Mg = torch.as_tensor(M, dtype=torch.float32, device="cuda")
    tg = torch.as_tensor(th, dtype=torch.float64, device="cuda")
    n = M.shape[0]
    r0 = max(norms_r0(M, th), 1e-300)

    def resid(x):
        F, lam, norms = solver.step_dense(Mg, x, theta=tg, precision="fp16x3")
        return F - x, lam, norms

    Z = torch.eye(n, dtype=torch.float32, device="cuda")
    Zp = fp = None
    incs, lams, xs, ts = [], [], [], []
    for _ in range(max_steps):
        f, lam, norms = resid(Z)
        rho = norms["residual_abs"] / r0
        if not np.isfinite(rho) or rho > 1e6 or rho <= tol:
            break
        incs.append((f.double().norm(dim=0) / Z.double().norm(dim=0)).float())
        lams.append(lam.double())
        if fp is None or len(incs) < 3:  # Picard steps until three histories are known
            Zp, fp = Z, f
            Z = Z + f
            continue
        dz, df = Z - Zp, f - fp
        gl = gamma_ls(f, fp)
        g_a = gl.clamp(-GAMMA_CLIP, GAMMA_CLIP).float()
        r_a = f - g_a[None, :] * df
        y_a = Z - g_a[None, :] * dz
        fa, _, _ = resid(y_a + r_a)
        fpic, _, _ = resid(Z + f)
        use_a = fa.double().norm(dim=0) < fpic.double().norm(dim=0)
        gamma = torch.where(use_a, g_a, torch.zeros_like(g_a))
        r = torch.where(use_a[None, :], r_a, f).double()
        Jr = torch.where(use_a[None, :], fa - r_a, fpic - f).double()
        num = -(r * Jr).sum(0)
        den = (Jr * Jr).sum(0)
        alpha = torch.where(den > 0, num / torch.where(den > 0, den, torch.ones_like(den)),
                            torch.ones_like(den)).clamp(0.05, 2.0).float()
        x6 = damping_features(torch.stack(incs[-3:]), torch.stack(lams[-3:])).float()
        xs.append(torch.cat([x6, gl.clamp(-4.0, 4.0).float()[:, None]], dim=1))
        ts.append(torch.stack([alpha, gamma], dim=1))
        Zn = Z + alpha[None, :] * f - gamma[None, :] * (dz + alpha[None, :] * df)
        Zp, fp = Z, f
        Z = Zn
    return xs, ts


def init_params(seed):
    """Uniform +-1/sqrt(fan_in) initial weights, FP16 (W1, b1, W2, b2, W3, b3)."""
    g = np.random.default_rng(seed)
    ni, nh, no = 7, 64, 2
    parts = [g.uniform(-1, 1, (ni, nh)) / np.sqrt(ni), g.uniform(-1, 1, nh) / np.sqrt(ni),
             g.uniform(-1, 1, (nh, nh)) / np.sqrt(nh), g.uniform(-1, 1, nh) / np.sqrt(nh),
             g.uniform(-1, 1, (nh, no)) / np.sqrt(nh), g.uniform(-1, 1, no) / np.sqrt(nh)]
    return np.concatenate([x.reshape(-1) for x in parts]).astype(np.float16)


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
            ipt.mixing_grad(p16, X[idx].contiguous(), T[idx].contiguous(), grad, loss)
            step += 1
            ipt.mixing_adam(master, p16, grad, m, v, lr, step)
            nb += 1
        print(f"epoch {ep}: mse {loss.item() / nb:.5f}", flush=True)
    return p16


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
    keep = torch.isfinite(X).all(1) & torch.isfinite(T).all(1)
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
