"""The bounded device-side waits of the tensor-core kernels give up instead of hanging: a wait
on a barrier that nothing completes (glv_check_bounded_wait, a short limit) ends, records
GLV_ERR_TIMEOUT in the status word, and leaves the context usable for the next call."""
import time

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def glv():
    from paper_2410_22347_gb300 import build_lib
    build_lib.build()
    from paper_2410_22347_gb300 import glv as g
    return g


def test_bounded_wait_times_out_and_reports(glv):
    dev = torch.device("cuda:0")
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    glv.glv_check_bounded_wait(20_000, st)  # 20 ms
    assert glv.glv_last_device_status(st) == glv.GLV_ERR_TIMEOUT
    waited = time.perf_counter() - t0
    assert 0.015 <= waited < 5.0, waited
    # the context is still usable: a projection right after runs and is correct
    rng = np.random.default_rng(0)
    Q = rng.standard_normal((300, 64)).astype(np.float32)
    A = rng.standard_normal((3, 16, 64)).astype(np.float32)
    st2 = torch.zeros(1, dtype=torch.int32, device=dev)
    Qp = glv.glv_project_queries(torch.from_numpy(Q).to(dev), torch.from_numpy(A).to(dev), glv.GLV_F32,
                                 d_status=st2)
    assert glv.glv_last_device_status(st2) == glv.GLV_OK
    ref = np.einsum("cdk,qk->qcd", A.astype(np.float64), Q.astype(np.float64))
    np.testing.assert_allclose(Qp.cpu().numpy(), ref, rtol=0, atol=1e-4 * np.abs(ref).max())


def test_bounded_wait_argument_checks(glv):
    st = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    with pytest.raises(glv.GlvError):
        glv.glv_check_bounded_wait(0, st)
    with pytest.raises(glv.GlvError):
        glv.glv_check_bounded_wait(2_000_000, st)
