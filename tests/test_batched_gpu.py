"""GPU parity of the batched solve (ipt_solve_batched) against the CPU oracle.

Each problem is Alg. 2 with all eigenpairs; the oracle solves the same
problem on its own.  FP32 arithmetic: fixed-iteration iterates within 2e-5 of
max |Z - E|, converged eigenvalues within 1e-5 relative, eigenvectors within
1e-4 of ||Z - E|| (rho <= 1e-6).
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2012_14702_gb300 import workloads as w

pytestmark = pytest.mark.gpu


def pack(mats):
    sizes = np.array([m.shape[0] for m in mats], dtype=np.int64)
    return sizes, np.concatenate([np.asarray(m, dtype=np.float64).reshape(-1) for m in mats])


def blocks(flat, sizes, square=True):
    out, o = [], 0
    for n in sizes:
        n = int(n)
        sz = n * n if square else n
        out.append(flat[o:o + sz])
        o += sz
    return out


SIZES = [1, 2, 3, 17, 31, 64, 65, 100, 130, 200, 257, 5, 96, 128, 129]


def small_batch(seed=21, scale=2e-2):
    g = w.rng(seed)
    mats = []
    for n in SIZES:
        a = g.standard_normal((n, n)) * scale / np.sqrt(n)
        a = np.triu(a, 1)
        a = a + a.T
        a[np.diag_indices(n)] = np.arange(1, n + 1) * 1.0
        mats.append(a)
    return mats


@pytest.mark.parametrize("m", [1, 2, 4])
def test_batched_fixed_iterations_match_oracle_iterates(ipt, m):
    mats = small_batch()
    sizes, flat = pack(mats)
    lam, Z, status, iters, info = ipt.Solver().solve_batched(
        sizes, torch.as_tensor(flat, dtype=torch.float32, device="cuda"), tol=0.0, max_iter=m,
        stop="increment")
    st, it = status.cpu().numpy(), iters.cpu().numpy()
    Zs = blocks(Z.cpu().numpy(), sizes)
    lams = blocks(lam.cpu().numpy(), sizes, square=False)
    for p, M in enumerate(mats):
        n = M.shape[0]
        # with tol = 0 a problem stops early only if its FP32 increment is exactly 0
        # (n = 1 at once; tiny n once converged to FP32 resolution)
        ref = oracle.ipt_solve(M, tol=0.0, max_iter=int(it[p]), stop="increment",
                               history=True)
        if st[p] == oracle.OK:
            assert it[p] <= m and ref["inc_hist"][-1] <= 1e-6, (p, n, it[p])
        else:
            assert st[p] == oracle.MAXITER and it[p] == m, (p, n, st[p], it[p])
        Zg = Zs[p].reshape(n, n).T  # column-major block
        scale = max(np.max(np.abs(ref["Z"] - np.eye(n))), 1e-30)
        assert np.max(np.abs(Zg - ref["Z"])) <= 2e-5 * scale + 1e-7, (p, n)
        np.testing.assert_allclose(lams[p], ref["lam"], rtol=1e-6, atol=1e-6)


def test_batched_converged_match_oracle_and_theta_forms(ipt):
    mats = small_batch(seed=22)
    sizes, flat = pack(mats)
    Mg = torch.as_tensor(flat, dtype=torch.float32, device="cuda")
    theta = np.concatenate([np.diag(M) for M in mats])
    s = ipt.Solver()
    lam, Z, status, iters, info = s.solve_batched(sizes, Mg, tol=1e-6, max_iter=50)
    assert info["status"] == "OK", info
    lam2, Z2, _, _, _ = s.solve_batched(sizes, Mg, theta=torch.as_tensor(theta, device="cuda"),
                                        tol=1e-6, max_iter=50)
    assert torch.equal(lam, lam2) and torch.equal(Z, Z2)
    Zs = blocks(Z.cpu().numpy(), sizes)
    lams = blocks(lam.cpu().numpy(), sizes, square=False)
    its = iters.cpu().numpy()
    for p, M in enumerate(mats):
        n = M.shape[0]
        ref = oracle.ipt_solve(M, tol=1e-13, max_iter=100)
        assert ref["status"] == oracle.OK
        np.testing.assert_allclose(lams[p], ref["lam"], rtol=1e-5)
        if n > 1:
            E = np.eye(n)
            err = np.linalg.norm(Zs[p].reshape(n, n).T - ref["Z"]) / np.linalg.norm(ref["Z"] - E)
            assert err <= 1e-4, (p, err)
        # the residual-stopped oracle takes the same number of evaluations
        ref6 = oracle.ipt_solve(M, tol=1e-6, max_iter=50, stop="residual")
        assert abs(int(its[p]) - ref6["iterations"]) <= 1, (p, its[p], ref6["iterations"])


@pytest.mark.parametrize("precision", ["f32", "bf16x3"])
def test_batched_per_problem_statuses(ipt, precision):
    mats = small_batch(seed=23)
    # problem 3 degenerate (repeated theta), problem 7 far outside the domain
    th = [np.diag(M).copy() for M in mats]
    th[3][1] = th[3][0]
    big = mats[7].copy()
    n7 = big.shape[0]
    big += (np.ones((n7, n7)) - np.eye(n7)) * 5.0
    mats[7] = big
    sizes, flat = pack(mats)
    lam, Z, status, iters, info = ipt.Solver().solve_batched(
        sizes, torch.as_tensor(flat, dtype=torch.float32, device="cuda"),
        theta=torch.as_tensor(np.concatenate(th), device="cuda"), tol=1e-6, max_iter=60,
        precision=precision)
    st = status.cpu().numpy()
    assert st[3] == oracle.DEGENERATE_THETA
    assert st[7] in (oracle.DIVERGED, oracle.MAXITER)
    others = [p for p in range(len(mats)) if p not in (3, 7)]
    assert np.all(st[others] == oracle.OK)
    assert info["status"] == "DEGENERATE_THETA"  # the first failing problem by index


def test_batched_argument_errors(ipt):
    s = ipt.Solver()
    M = torch.zeros(1025 * 1025, dtype=torch.float32, device="cuda")
    *_, info = s.solve_batched([1025], M)
    assert info["status"] == "INVALID_ARG"
    with pytest.raises(ValueError):
        s.solve_batched([3, 4], torch.zeros(10, dtype=torch.float32, device="cuda"))


def test_batched_full_size_sampled_problems(ipt):
    """The batched configuration: 4096 problems, n_p ~ U{32..512}, theta_i = i,
    N(0,1)*0.01/sqrt(n_p) symmetric perturbations, seed 4; every problem reaches
    rho <= 1e-6 and sampled problems match the oracle."""
    count, nmin, nmax, scale, seed = w.BATCHED_CONFIGS["batched_4096_n32_512"]
    sizes, flat, th = w.batched_dense(count, nmin, nmax, scale, seed)
    lam, Z, status, iters, info = ipt.Solver().solve_batched(
        sizes, torch.as_tensor(flat, device="cuda"), tol=1e-6, max_iter=30)
    assert info["status"] == "OK", info
    offs = np.concatenate([[0], np.cumsum(sizes * sizes)])
    voffs = np.concatenate([[0], np.cumsum(sizes)])
    for p in [0, 1, 77, 1000, 2047, 3333, 4095, int(np.argmax(sizes))]:
        n = int(sizes[p])
        M = flat[offs[p]:offs[p + 1]].astype(np.float64).reshape(n, n)
        ref = oracle.ipt_solve(M, th[voffs[p]:voffs[p + 1]], tol=1e-13, max_iter=100)
        lg = lam[voffs[p]:voffs[p + 1]].cpu().numpy()
        np.testing.assert_allclose(lg, ref["lam"], rtol=1e-5)
        Zg = Z[offs[p]:offs[p + 1]].cpu().numpy().reshape(n, n).T
        err = np.linalg.norm(Zg - ref["Z"]) / np.linalg.norm(ref["Z"] - np.eye(n))
        assert err <= 1e-4, (p, err)


def test_batched_largest_orders(ipt):
    """Orders up to the 1024 limit in one batch (scratch sized by the largest)."""
    mats = []
    g = w.rng(31)
    for n in [1024, 700, 1, 513]:
        a = g.standard_normal((n, n)) * 1e-2 / np.sqrt(n)
        a = np.triu(a, 1)
        a = a + a.T
        a[np.diag_indices(n)] = np.arange(1, n + 1) * 1.0
        mats.append(a)
    sizes, flat = pack(mats)
    lam, Z, status, iters, info = ipt.Solver().solve_batched(
        sizes, torch.as_tensor(flat, dtype=torch.float32, device="cuda"), tol=1e-6, max_iter=30)
    assert info["status"] == "OK", info
    Zs = blocks(Z.cpu().numpy(), sizes)
    lams = blocks(lam.cpu().numpy(), sizes, square=False)
    for p, M in enumerate(mats):
        n = M.shape[0]
        ref = oracle.ipt_solve(M, tol=1e-13, max_iter=100)
        np.testing.assert_allclose(lams[p], ref["lam"], rtol=1e-5)
        if n > 1:
            err = np.linalg.norm(Zs[p].reshape(n, n).T - ref["Z"]) / np.linalg.norm(
                ref["Z"] - np.eye(n))
            assert err <= 1e-4, (p, err)


def test_batched_tiles_give_identical_iterates(ipt):
    """Both output tiles accumulate every product entry in the same order: forced
    32 and 64 tiles give bit-identical fixed-iteration iterates, which match the
    oracle."""
    mats = small_batch(seed=24)
    sizes, flat = pack(mats)
    Mg = torch.as_tensor(flat, dtype=torch.float32, device="cuda")
    outs = []
    for tiles in [(32, 32, 32), (64, 64, 64), (32, 64, 32)]:
        s = ipt.Solver()
        s.batched_tiles = tiles
        lam, Z, status, iters, _ = s.solve_batched(sizes, Mg, tol=0.0, max_iter=3,
                                                   stop="increment")
        assert s.batched_tiles == tiles
        outs.append((lam, Z, iters))
    for lam, Z, iters in outs[1:]:
        assert torch.equal(lam, outs[0][0]) and torch.equal(Z, outs[0][1])
        assert torch.equal(iters, outs[0][2])
    Zs = blocks(outs[0][1].cpu().numpy(), sizes)
    its = outs[0][2].cpu().numpy()
    for p in [4, 9, 10]:
        M, n = mats[p], mats[p].shape[0]
        ref = oracle.ipt_solve(M, tol=0.0, max_iter=int(its[p]), stop="increment")
        scale = max(np.max(np.abs(ref["Z"] - np.eye(n))), 1e-30)
        assert np.max(np.abs(Zs[p].reshape(n, n).T - ref["Z"])) <= 2e-5 * scale + 1e-7


def test_batched_autotuner_tunes_the_classes_met(ipt):
    s = ipt.Solver()
    assert s.batched_tiles == (0, 0, 0)
    mats = small_batch(seed=25)  # orders up to 257: classes 0, 1 and 2
    sizes, flat = pack(mats[:8])  # orders <= 100: classes 0 and 1 only
    Mg = torch.as_tensor(flat, dtype=torch.float32, device="cuda")
    *_, info = s.solve_batched(sizes, Mg, tol=1e-6, max_iter=50)
    assert info["status"] == "OK"
    t = s.batched_tiles
    assert t[0] in (32, 64) and t[1] in (32, 64) and t[2] == 0, t
    with pytest.raises(ValueError):
        s.batched_tiles = (48, 64, 64)
    assert s.batched_tiles == t


@pytest.mark.parametrize("precision", ["f32", "bf16x3"])
def test_batched_graph_replay_reads_current_inputs(ipt, precision):
    """The captured graph is replayed while orders, pointers and tolerances
    repeat: new contents of the same buffers give that batch's solution, and a
    changed tolerance is captured anew."""
    a = small_batch(seed=26)
    b = small_batch(seed=27)
    sizes, fa = pack(a)
    _, fb = pack(b)
    s = ipt.Solver()
    Mg = torch.as_tensor(fa, dtype=torch.float32, device="cuda")
    lam_a, Z_a, *_ = [x.clone() if torch.is_tensor(x) else x
                      for x in s.solve_batched(sizes, Mg, tol=1e-6, max_iter=50,
                                               precision=precision)]
    Mg.copy_(torch.as_tensor(fb, dtype=torch.float32))
    lam_b, Z_b, _, _, info = s.solve_batched(sizes, Mg, tol=1e-6, max_iter=50,
                                             precision=precision)
    assert info["status"] == "OK"
    fresh = ipt.Solver()
    fresh.batched_tiles = s.batched_tiles
    lam_r, Z_r, *_ = fresh.solve_batched(sizes, torch.as_tensor(fb, dtype=torch.float32,
                                                               device="cuda"), tol=1e-6,
                                         max_iter=50, precision=precision)
    assert torch.equal(lam_b, lam_r) and not torch.equal(lam_a, lam_b)
    lam_c, _, _, iters_c, info = s.solve_batched(sizes, Mg, tol=0.0, max_iter=2,
                                                 stop="increment", precision=precision)
    assert info["iterations"] <= 2 and int(iters_c.max()) == 2
    lams = blocks(lam_b.cpu().numpy(), sizes, square=False)
    for p in [3, 12]:
        ref = oracle.ipt_solve(b[p], tol=1e-13, max_iter=100)
        np.testing.assert_allclose(lams[p], ref["lam"], rtol=1e-5)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_batched_bf16x3_tensor_core_iterates_match_oracle(ipt, m):
    """The tensor-core variant (split BF16 x3 products in 128 x 128 tiles): the
    iterates of a fixed number of evaluations within 2e-5 of max |Z - E| of the
    oracle's (the product's relative error is ~2^-16)."""
    mats = small_batch(seed=28)
    sizes, flat = pack(mats)
    lam, Z, status, iters, info = ipt.Solver().solve_batched(
        sizes, torch.as_tensor(flat, dtype=torch.float32, device="cuda"), tol=0.0, max_iter=m,
        stop="increment", precision="bf16x3")
    st, it = status.cpu().numpy(), iters.cpu().numpy()
    Zs = blocks(Z.cpu().numpy(), sizes)
    lams = blocks(lam.cpu().numpy(), sizes, square=False)
    for p, M in enumerate(mats):
        n = M.shape[0]
        ref = oracle.ipt_solve(M, tol=0.0, max_iter=int(it[p]), stop="increment")
        if st[p] != oracle.OK:
            assert st[p] == oracle.MAXITER and it[p] == m, (p, n, st[p], it[p])
        Zg = Zs[p].reshape(n, n).T
        scale = max(np.max(np.abs(ref["Z"] - np.eye(n))), 1e-30)
        assert np.max(np.abs(Zg - ref["Z"])) <= 2e-5 * scale + 1e-7, (p, n)
        np.testing.assert_allclose(lams[p], ref["lam"], rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("precision,tol", [("bf16x3", 1e-6), ("bf16", 1e-4)])
def test_batched_tensor_core_converged_match_oracle(ipt, precision, tol):
    mats = small_batch(seed=29) + [np.diag(np.arange(1.0, 301.0))]
    g = w.rng(30)
    for n in [384, 513]:
        a = g.standard_normal((n, n)) * 1e-2 / np.sqrt(n)
        a = np.triu(a, 1)
        a = a + a.T
        a[np.diag_indices(n)] = np.arange(1, n + 1) * 1.0
        mats.append(a)
    sizes, flat = pack(mats)
    lam, Z, status, iters, info = ipt.Solver().solve_batched(
        sizes, torch.as_tensor(flat, dtype=torch.float32, device="cuda"), tol=tol, max_iter=60,
        precision=precision)
    assert info["status"] == "OK", (info, status.cpu().numpy())
    Zs = blocks(Z.cpu().numpy(), sizes)
    lams = blocks(lam.cpu().numpy(), sizes, square=False)
    for p, M in enumerate(mats):
        n = M.shape[0]
        ref = oracle.ipt_solve(M, tol=1e-13, max_iter=100)
        np.testing.assert_allclose(lams[p], ref["lam"], rtol=1e-5 if tol < 1e-5 else 1e-4)
        if n > 1 and np.any(ref["Z"] != np.eye(n)):
            err = np.linalg.norm(Zs[p].reshape(n, n).T - ref["Z"]) / np.linalg.norm(
                ref["Z"] - np.eye(n))
            assert err <= (1e-4 if tol < 1e-5 else 1e-2), (p, n, err)


def test_batched_bf16x3_full_size_configuration(ipt):
    count, nmin, nmax, scale, seed = w.BATCHED_CONFIGS["batched_4096_n32_512"]
    sizes, flat, th = w.batched_dense(count, nmin, nmax, scale, seed)
    lam, Z, status, iters, info = ipt.Solver().solve_batched(
        sizes, torch.as_tensor(flat, device="cuda"), tol=1e-6, max_iter=30, precision="bf16x3")
    assert info["status"] == "OK", info
    offs = np.concatenate([[0], np.cumsum(sizes * sizes)])
    voffs = np.concatenate([[0], np.cumsum(sizes)])
    for p in [0, 5, 2048, 4095, int(np.argmax(sizes))]:
        n = int(sizes[p])
        M = flat[offs[p]:offs[p + 1]].astype(np.float64).reshape(n, n)
        ref = oracle.ipt_solve(M, th[voffs[p]:voffs[p + 1]], tol=1e-13, max_iter=100)
        np.testing.assert_allclose(lam[voffs[p]:voffs[p + 1]].cpu().numpy(), ref["lam"],
                                   rtol=1e-5)
        Zg = Z[offs[p]:offs[p + 1]].cpu().numpy().reshape(n, n).T
        assert np.linalg.norm(Zg - ref["Z"]) / np.linalg.norm(ref["Z"] - np.eye(n)) <= 1e-4


@pytest.mark.parametrize("precision", ["f32", "bf16x3"])
def test_batched_largest_orders_converge(ipt, precision):
    """The largest order the batched solve takes (1024: eight 128-row blocks and
    sixteen 64-deep slices per product on the tensor cores) beside ragged orders
    just under it and a tiny one, converged to rho <= 1e-6 against the oracle."""
    g = w.rng(41)
    mats = []
    for n in [1024, 1023, 897, 3]:
        a = g.standard_normal((n, n)) * 1e-2 / np.sqrt(n)
        a = np.triu(a, 1)
        a = a + a.T
        a[np.diag_indices(n)] = np.arange(1, n + 1) * 1.0
        mats.append(a)
    sizes, flat = pack(mats)
    lam, Z, status, iters, info = ipt.Solver().solve_batched(
        sizes, torch.as_tensor(flat, dtype=torch.float32, device="cuda"), tol=1e-6, max_iter=40,
        precision=precision)
    assert info["status"] == "OK", (info, status.cpu().numpy())
    Zs = blocks(Z.cpu().numpy(), sizes)
    lams = blocks(lam.cpu().numpy(), sizes, square=False)
    for p, M in enumerate(mats):
        n = M.shape[0]
        ref = oracle.ipt_solve(M, tol=1e-13, max_iter=100)
        np.testing.assert_allclose(lams[p], ref["lam"], rtol=1e-5)
        err = np.linalg.norm(Zs[p].reshape(n, n).T - ref["Z"]) / np.linalg.norm(ref["Z"] - np.eye(n))
        assert err <= 1e-4, (p, n, err)
