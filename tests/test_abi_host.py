"""CPU checks of the C ABI: the library loads, exports every entry point the header
declares, and rejects invalid arguments on the host before touching the GPU."""
import ctypes
import os
import re

import pytest

from paper_2410_22347_gb300 import build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "glv.h")


@pytest.fixture(scope="module")
def lib():
    path = build_lib.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(glv_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_search_path():
    names = declared_functions()
    for fn in ("glv_build_reduced", "glv_project_queries", "glv_score_candidates", "glv_topk",
               "glv_rerank", "glv_assign_tags"):
        assert fn in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert names
    for fn in names:
        assert hasattr(lib, fn), f"{fn} declared in glv.h but not exported"


P = ctypes.c_void_p
FAKE = P(4096)   # never dereferenced: validation rejects before any CUDA call
INV = 1


def _ret_i32(lib, name, argtypes):
    f = getattr(lib, name)
    f.restype = ctypes.c_int32
    f.argtypes = argtypes
    return f


def test_host_validation_rejects_bad_arguments(lib):
    i64, i32 = ctypes.c_int64, ctypes.c_int32
    lib.glv_abi_version.restype = i32
    assert lib.glv_abi_version() == 4
    lib.glv_min_row_stride.restype = i64
    lib.glv_min_row_stride.argtypes = [i32, i32]
    assert lib.glv_min_row_stride(160, 0) == 640
    assert lib.glv_min_row_stride(160, 1) == 320
    assert lib.glv_min_row_stride(127, 2) == 128
    assert lib.glv_min_row_stride(3, 1) == 16
    assert lib.glv_min_row_stride(0, 0) == -1

    topk = _ret_i32(lib, "glv_topk", [P, P, P, i64, i32, P, P, P])
    assert topk(FAKE, FAKE, FAKE, 4, 0, FAKE, FAKE, None) == INV          # kappa = 0
    assert topk(FAKE, FAKE, FAKE, 4, 1025, FAKE, FAKE, None) == INV       # kappa > max
    assert topk(None, FAKE, FAKE, 4, 10, FAKE, FAKE, None) == INV         # null scores
    assert topk(None, None, None, 0, 10, None, None, None) == 0           # empty: nothing to do

    rerank = _ret_i32(lib, "glv_rerank", [P, i64, i32, P, i64, P, i32, i32, P, P, P, P])
    assert rerank(FAKE, 10, 8, FAKE, 2, FAKE, 5, 6, FAKE, FAKE, None, None) == INV   # k > kappa
    assert rerank(FAKE, 10, 0, FAKE, 2, FAKE, 5, 2, FAKE, FAKE, None, None) == INV   # D = 0
    assert rerank(FAKE, 10, 8, None, 2, FAKE, 5, 2, FAKE, FAKE, None, None) == INV   # null Q

    build = _ret_i32(lib, "glv_build_reduced", [P, i64, i32, P, P, i32, i32, i32, P, i64, P, P, P, P])
    ok_args = dict(X=FAKE, N=100, D=64, tags=FAKE, B=FAKE, C=4, d=16, dt=0, Xred=FAKE, rs=64,
                   scales=None, ws=P(4096 * 256), st=None)

    def b(**kw):
        a = dict(ok_args, **kw)
        return build(a["X"], a["N"], a["D"], a["tags"], a["B"], a["C"], a["d"], a["dt"], a["Xred"],
                     a["rs"], a["scales"], a["ws"], None, a["st"])
    assert b(d=65) == INV                  # d > D
    assert b(rs=48) == INV                 # stride below d * 4
    assert b(rs=72) == INV                 # stride not a multiple of 16
    assert b(dt=2) == INV                  # FP8 without scales
    assert b(dt=1, scales=FAKE) == INV     # scales given for BF16
    assert b(dt=7) == INV                  # unknown dtype
    assert b(C=0) == INV
    assert b(C=70000) == INV
    assert b(Xred=P(4096 + 8)) == INV      # misaligned store
    assert b(ws=P(4096 + 64)) == INV       # misaligned workspace
    assert b(N=0) == 0                     # empty database: nothing to do

    score = _ret_i32(lib, "glv_score_candidates", [P, i64, i32, i32, P, i64, P, i32, P, i64, P, P, P, P, P])
    assert score(FAKE, 3, 4, 16, FAKE, 32, None, 0, FAKE, 10, FAKE, FAKE, FAKE, None, None) == INV  # stride
    assert score(FAKE, 3, 4, 16, FAKE, 64, None, 2, FAKE, 10, FAKE, FAKE, FAKE, None, None) == INV  # fp8, no scales
    assert score(FAKE, 3, 0, 16, FAKE, 64, None, 0, FAKE, 10, FAKE, FAKE, FAKE, None, None) == INV  # C = 0
    assert score(FAKE, 3, 4, 16, FAKE, 64, None, 0, FAKE, 10, None, FAKE, FAKE, None, None) == INV  # null off
    assert score(FAKE, 3, 65536, 1024, FAKE, 4096, None, 0, FAKE, 10, FAKE, FAKE, FAKE, None, None) == 3  # too big for smem

    proj = _ret_i32(lib, "glv_project_queries", [P, i64, i32, P, i32, i32, i32, P, P, P, P])
    assert proj(FAKE, 5, 32, FAKE, 2, 33, 0, FAKE, None, None, None) == INV   # d > D
    assert proj(FAKE, 5, 32, FAKE, 2, 8, 2, FAKE, None, None, None) == INV    # FP8 compute not offered
    assert proj(FAKE, 5, 32, None, 2, 8, 0, FAKE, None, None, None) == INV
    assert proj(FAKE, 5, 32, FAKE, 2, 8, 1, FAKE, None, None, None) == INV    # BF16 needs a workspace
    assert proj(FAKE, 5, 32, FAKE, 2, 8, 1, FAKE, P(4096 + 16), None, None) == INV  # misaligned workspace
    lib.glv_project_queries_workspace_size.restype = ctypes.c_size_t
    lib.glv_project_queries_workspace_size.argtypes = [i64, i32, i32, i32, i32]
    # BF16: (nq + C*d) rows x 64-padded K x 2 bytes, each operand rounded to 1 KB
    assert lib.glv_project_queries_workspace_size(10000, 768, 32, 160, 1) == 10000 * 768 * 2 + 5120 * 768 * 2
    # FP32 (TF32 hi/lo): K padded to 128; Q 100 x 128 x 4 B and A 16 x 128 x 4 B, two copies each
    assert lib.glv_project_queries_workspace_size(100, 100, 2, 8, 0) == 2 * 51200 + 2 * 8192

    lib.glv_score_topk_workspace_size.restype = ctypes.c_size_t
    lib.glv_score_topk_workspace_size.argtypes = [i64, i64]
    # header 256 B + chunk_start (nq + 1) + done (nq) + a 24-byte record per work item (one per
    # query and per 4096 candidates, plus one), each array rounded to 256 bytes
    r256 = lambda b: (b + 255) // 256 * 256
    assert lib.glv_score_topk_workspace_size(10000, 20480000) == \
        256 + r256(10001 * 4) + r256(10000 * 4) + r256((10000 + 5000 + 1) * 24)
    stk = _ret_i32(lib, "glv_score_topk", [P, i64, i32, i32, P, i64, P, i32, P, i64, P, P, i64, i32, P, P, P, P, P, P])
    args = [FAKE, 700, 4, 16, FAKE, 64, None, 0, FAKE, 10, FAKE, FAKE, 1000, 10, FAKE]
    assert stk(*args, None, FAKE, FAKE, None, None) == INV              # no workspace
    assert stk(*args, P(4096 + 16), FAKE, FAKE, None, None) == INV      # misaligned workspace
    bad = list(args)
    bad[12] = -1
    assert stk(*bad, FAKE, FAKE, FAKE, None, None) == INV               # negative candidate count

    lib.glv_search_workspace_size.restype = ctypes.c_size_t
    lib.glv_search_workspace_size.argtypes = [i64, i32, i32, i32, i32, i64, i32]
    # Qp + projection operands + score scratch + work plan + kappa survivors, each 256-aligned
    want = (r256(10000 * 32 * 160 * 4) + r256(10000 * 768 * 2 + 5120 * 768 * 2) + r256(20480000 * 4)
            + r256(256 + r256(10001 * 4) + r256(10000 * 4) + r256((10000 + 5000 + 1) * 24)) + r256(10000 * 100 * 8))
    assert lib.glv_search_workspace_size(10000, 768, 32, 160, 1, 20480000, 100) == want
    assert lib.glv_search_workspace_size(10000, 768, 32, 160, 1, 20480000, 0) == want - r256(10000 * 100 * 8)
    assert lib.glv_search_workspace_size(10, 0, 32, 160, 1, 100, 10) == 0        # D = 0
    search = _ret_i32(lib, "glv_search", [P, i64, i32, P, i64, P, i32, i32, i32, P, i64, P, i32, P, P, P, i64,
                                          i32, i32, P, P, P, P, P])
    head = [FAKE, 1000, 64, FAKE, 5, FAKE, 4, 16, 1, FAKE, 64, None, 1, FAKE, FAKE, FAKE, 500]

    def srch(kappa, k, ws=FAKE, compute=1, nq=5):
        a = list(head)
        a[4], a[8] = nq, compute
        return search(*a, kappa, k, ws, FAKE, FAKE, None, None)
    assert srch(8, 10) == INV               # kappa below k
    assert srch(10, 0) == INV               # k = 0
    assert srch(2000, 10) == INV            # kappa beyond the maximum
    assert srch(20, 10, compute=2) == INV   # FP8 projection not offered
    assert srch(20, 10, ws=None) == INV     # no workspace
    assert srch(20, 10, ws=P(4096 + 64)) == INV  # misaligned workspace
    assert srch(20, 10, nq=0) == 0          # no queries: nothing to do

    tags = _ret_i32(lib, "glv_assign_tags", [P, i64, i32, P, i32, P, P, P])
    assert tags(FAKE, 10, 8, FAKE, 0, FAKE, None, None) == INV
    assert tags(FAKE, 10, 2048, FAKE, 4, FAKE, None, None) == 3          # D beyond the kernel's limit

    lib.glv_status_string.restype = ctypes.c_char_p
    assert lib.glv_status_string(2) == b"id or tag out of range"
    lds = _ret_i32(lib, "glv_last_device_status", [P, P])
    assert lds(None, None) == INV           # no status word: rejected before any CUDA call

    # scoring configuration: host-only state, checked without a GPU
    setc = _ret_i32(lib, "glv_set_score_config", [i32, i32, i32, i32, i32])
    getc = _ret_i32(lib, "glv_get_score_config", [i32, i32, P, P, P, P])
    g, m, c, h = i32(0), i32(0), i32(0), i32(0)
    ref = [ctypes.byref(x) for x in (g, m, c, h)]
    assert setc(1, 4, 1, 164, 0) == 0
    assert getc(1, 160, *ref) == 0 and (g.value, m.value, c.value, h.value) == (4, 1, 164, 0)
    assert setc(1, 4, 1, 8, 1) == INV       # carveout cap below 16 KB
    assert setc(1, 4, 1, 300, 1) == INV     # above the SM's shared memory
    assert setc(1, 3, 0, 0, 1) == INV       # lanes per candidate not a power of two
    assert setc(1, 4, 3, 0, 1) == INV       # no gather mode 3
    assert setc(1, 4, 0, 0, 8) == INV       # schedules are 0..7
    assert setc(1, 4, 0, 0, 3) == 0         # wide CTAs, planned items
    assert getc(1, 160, *ref) == 0 and (g.value, m.value, h.value) == (4, 0, 3)
    assert setc(1, 16, 0, 0, 3) == 0        # no wide kernel with 16 lanes: the bit is dropped
    assert getc(1, 160, *ref) == 0 and (g.value, h.value) == (16, 1)
    assert setc(5, 4, 0, 0, 1) == INV       # unknown store type
    assert getc(1, 160, None, *ref[1:]) == INV
    assert setc(1, 0, 0, 0, 1) == 0
    assert getc(1, 160, *ref) == 0 and c.value == 0 and h.value == 1


def test_product_path_has_no_oracle_dependency():
    """The CUDA library and its binding never import, link or load the oracle."""
    pkg = os.path.join(ROOT, "paper_2410_22347_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")) and f != "synth.py":
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "glv_oracle" not in text and "liboracle" not in text, f
