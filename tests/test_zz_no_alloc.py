"""glv_build_reduced_noalloc: the reduced-store build for callers that cannot allocate
device memory (their memory is owned by a host framework's pool or a fixed budget, or
cudaMalloc's device synchronisation is not acceptable on their path).  It takes only
inputs and outputs and keeps its scratch in a fixed device array inside the library.

These tests call it through the C ABI and check it against glv_build_reduced (which takes
a caller-provided workspace), byte for byte (the same kernels run on the same inputs), on
two calls in a row with different shapes and cluster layouts, so that scratch left over from
the first call cannot leak into the second.  The file is named to be collected last.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def glv():
    from paper_2410_22347_gb300 import build_lib
    build_lib.build()
    from paper_2410_22347_gb300 import glv as g
    return g


def _problem(seed, N, D, d, C, skew):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, D)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    B = (rng.standard_normal((C, d, D)) / np.sqrt(D)).astype(np.float32)
    if skew:   # most rows in one cluster, some clusters empty
        tags = np.where(rng.random(N) < 0.8, 1, rng.integers(0, C, N)).astype(np.uint16)
        tags[tags == C - 2] = C - 1
    else:
        tags = rng.integers(0, C, N).astype(np.uint16)
    dev = torch.device("cuda:0")
    return (torch.from_numpy(X).to(dev), torch.from_numpy(tags).to(dev), torch.from_numpy(B).to(dev),
            np.linalg.norm(B, axis=2)[tags] * np.linalg.norm(X, axis=1)[:, None])


def _decode(glv, raw, dt, d, scales):
    raw = raw.cpu().numpy()
    if dt == glv.GLV_F32:
        return raw.view(np.float32)[:, :d].astype(np.float64)
    if dt == glv.GLV_BF16:
        v = raw.view(np.uint16)[:, :d].astype(np.uint32) << 16
        return v.view(np.float32).astype(np.float64)
    codes = torch.from_numpy(np.ascontiguousarray(raw[:, :d])).view(torch.float8_e4m3fn).to(torch.float64)
    return codes.numpy() * scales.cpu().numpy().astype(np.float64)[:, None]


@pytest.mark.parametrize("first,second", [
    (dict(seed=1, N=5000, D=96, d=27, C=7, skew=False, dt="f32"),
     dict(seed=2, N=3001, D=128, d=40, C=12, skew=True, dt="f32")),
    (dict(seed=3, N=20000, D=256, d=64, C=33, skew=True, dt="bf16"),
     dict(seed=4, N=777, D=64, d=16, C=5, skew=False, dt="fp8")),
])
def test_noalloc_matches_workspace_build_twice(glv, first, second):
    for case in (first, second):
        X, tags, B, scale = _problem(case["seed"], case["N"], case["D"], case["d"], case["C"], case["skew"])
        dt = glv.DTYPES[case["dt"]]
        d = case["d"]
        rs = glv.min_row_stride(d, dt)
        ref, ref_sc = glv.glv_build_reduced(X, tags, B, dt)
        out = torch.full((case["N"], rs), 0x5A, dtype=torch.uint8, device=X.device)
        sc = torch.empty(case["N"], dtype=torch.float32, device=X.device) if case["dt"] == "fp8" else None
        status = torch.zeros(1, dtype=torch.int32, device=X.device)
        glv.glv_build_reduced_noalloc(X, tags, B, dt, out, rs, sc, d_status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        # the same kernels on the same inputs (a row's result does not depend on where the
        # grouping put it): the stored bytes and the FP8 scales must be identical
        assert torch.equal(out[:, :d * glv.elem_bytes(dt)], ref[:, :d * glv.elem_bytes(dt)])
        if sc is not None:
            assert torch.equal(sc.view(torch.int32), ref_sc.view(torch.int32))
        got = _decode(glv, out, dt, d, sc)
        want = _decode(glv, ref, dt, d, ref_sc)
        assert np.all(np.abs(got - want) <= TOL * np.maximum(np.abs(want), scale))
        pad = out.cpu().numpy()[:, d * glv.elem_bytes(dt):rs]
        assert np.all(pad == 0)


def test_noalloc_rejects_sizes_beyond_its_scratch(glv):
    dev = torch.device("cuda:0")
    lib = glv.lib()
    import ctypes
    fake = ctypes.c_void_p(4096)
    # N above the maximum: rejected on the host before anything is enqueued
    st = lib.glv_build_reduced_noalloc(fake, (1 << 20) + 1, 64, fake, fake, 4, 16, glv.GLV_F32, fake, 64, None,
                                       None, None)
    assert st == glv.GLV_ERR_UNSUPPORTED
    st = lib.glv_build_reduced_noalloc(fake, 1000, 64, fake, fake, 4097, 16, glv.GLV_F32, fake, 64, None,
                                       None, None)
    assert st == glv.GLV_ERR_UNSUPPORTED
    del dev
