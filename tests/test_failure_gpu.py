"""The failure path of the device-side waits, on the GPU, without a fault or a hang.

Every wait of the tensor-core product kernel on a shared-memory barrier is bounded
in time; on expiry the kernel records a timeout and returns, and the solve reports
IPT_DEVICE_TIMEOUT.  ipt_check_bounded_wait runs that same wait on a barrier that
nothing completes (a flag that nothing sets): the wait must give up after its
limit, and the context must stay usable for the next solve.
"""

import numpy as np
import pytest
import torch

from paper_2012_14702_gb300 import workloads as w

pytestmark = pytest.mark.gpu


def test_bounded_wait_completes_when_the_barrier_is_completed(ipt):
    ok, waited = ipt.check_bounded_wait(True, limit_s=1.0)
    assert ok and waited < 0.5


def test_bounded_wait_gives_up_and_the_context_stays_usable(ipt):
    ok, waited = ipt.check_bounded_wait(False, limit_s=0.2)
    assert not ok
    assert 0.2 <= waited < 2.0, waited
    M, th = w.dense_symmetric(256, 0.02, 1, theta_step=1.0)
    lam, Z, info = ipt.Solver().solve_dense(
        torch.as_tensor(M, dtype=torch.float32, device="cuda"),
        theta=torch.as_tensor(th, device="cuda"), tol=1e-6, max_iter=50)
    assert info["status"] == "OK"
    np.testing.assert_allclose(np.sort(lam.cpu().numpy()), np.linalg.eigvalsh(M), rtol=1e-6)


def test_bounded_wait_argument_errors(ipt):
    for bad in [0.0, -1.0, 11.0]:
        with pytest.raises(RuntimeError):
            ipt.check_bounded_wait(False, limit_s=bad)
