"""Run repeated solves of one named workload (for profilers and quick checks).

    python -m paper_2012_14702_gb300.run_case dense_n8192_eps1e-3 --solves 3
    python -m paper_2012_14702_gb300.run_case csr_n2p20_k64 --solves 2

Each solve goes through the C ABI exactly as a user's call would (inputs
resident on the device); the line printed per solve gives its status,
evaluations, residual and wall time.  Under a kernel profiler, ``--solves``
and the kernel-name filter select which launches are captured.
"""

from __future__ import annotations

import argparse
import time

from paper_2012_14702_gb300 import workloads


def run_dense(name, solves, precision, tol):
    import torch
    from paper_2012_14702_gb300 import ipt
    n, step, scale, seed = workloads.DENSE_CONFIGS[name]
    M, th = workloads.dense_symmetric(n, scale, seed, theta_step=step)
    Mg = torch.as_tensor(M, dtype=torch.float32, device="cuda")
    thg = torch.as_tensor(th, dtype=torch.float64, device="cuda")
    del M
    s = ipt.Solver()
    for i in range(solves):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, info = s.solve_dense(Mg, theta=thg, tol=tol, max_iter=40, precision=precision)
        torch.cuda.synchronize()
        print(f"{name} solve {i}: {info['status']} iterations {info['iterations']} "
              f"rho {info['rho']:.3e} {1e3 * (time.perf_counter() - t0):.2f} ms", flush=True)
        if info["status"] != "OK":
            raise SystemExit(1)


def run_csr(name, solves, precision, tol, window=True):
    import torch
    from paper_2012_14702_gb300 import ipt
    n, per_row, band, scale, seed, k = workloads.CSR_CONFIGS[name]
    rowptr, colind, vals, th = workloads.csr_banded(n, per_row, band, scale, seed=seed)
    cols = workloads.lowest_columns(th, k)
    rp = torch.as_tensor(rowptr, device="cuda")
    ci = torch.as_tensor(colind, device="cuda")
    vv = torch.as_tensor(vals, dtype=torch.float32, device="cuda")
    cg = torch.as_tensor(cols, device="cuda")
    s = ipt.Solver()
    for i in range(solves):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, info = s.solve_csr(rp, ci, vv, n, cols=cg, tol=tol, max_iter=50,
                                 precision="f32" if precision == "staged" else precision,
                                 window=window)
        torch.cuda.synchronize()
        print(f"{name} solve {i}: {info['status']} iterations {info['iterations']} "
              f"rho {info['rho']:.3e} {1e3 * (time.perf_counter() - t0):.2f} ms", flush=True)
        if info["status"] != "OK":
            raise SystemExit(1)


def run_batched(name, solves, tol, tiles=None, precision="f32"):
    import torch
    from paper_2012_14702_gb300 import ipt
    count, nmin, nmax, scale, seed = workloads.BATCHED_CONFIGS[name]
    sizes, flat, _ = workloads.batched_dense(count, nmin, nmax, scale, seed)
    Mg = torch.as_tensor(flat, device="cuda")
    s = ipt.Solver()
    if tiles:
        s.batched_tiles = tiles  # fixed tiles: no tuning launches before the solves
    for i in range(solves):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, _, iters, info = s.solve_batched(sizes, Mg, tol=tol, max_iter=30,
                                               precision=precision)
        torch.cuda.synchronize()
        print(f"{name} solve {i}: {info['status']} evaluations {info['iterations']} (max) "
              f"{1e3 * (time.perf_counter() - t0):.2f} ms, tiles {s.batched_tiles}", flush=True)
        if info["status"] != "OK":
            raise SystemExit(1)


def main(argv=None):
    names = (sorted(workloads.DENSE_CONFIGS) + sorted(workloads.CSR_CONFIGS) +
             sorted(workloads.BATCHED_CONFIGS))
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("workload", choices=names)
    ap.add_argument("--solves", type=int, default=2)
    ap.add_argument("--precision", default="staged")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--all-rows", action="store_true",
                    help="sparse workloads: evaluate every row (no active window)")
    ap.add_argument("--tiles", default=None,
                    help="batched workloads: output tiles per size class, e.g. 64,64,64 "
                         "(default: tuned on the first solve)")
    a = ap.parse_args(argv)
    if a.workload in workloads.DENSE_CONFIGS:
        run_dense(a.workload, a.solves, a.precision, a.tol)
    elif a.workload in workloads.BATCHED_CONFIGS:
        tiles = [int(x) for x in a.tiles.split(",")] if a.tiles else None
        prec = a.precision if a.precision in ("bf16x3", "bf16") else "f32"
        run_batched(a.workload, a.solves, a.tol, tiles, prec)
    else:
        run_csr(a.workload, a.solves, a.precision, a.tol, window=not a.all_rows)


if __name__ == "__main__":
    main()
