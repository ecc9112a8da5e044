"""The whole search step captured in a CUDA graph (batching form: one persistent scoring
launch per step, replayed without host launches) gives, replay after replay, exactly the
results of the same calls launched eagerly.

Each replay runs on new queries and new candidate lists copied into the captured input
buffers.  The lists are lognormal-length (mean 1500, sigma 1.2, up to 20000 candidates), so
lists of 8192 or more are cut into work items whose top-kappa lists are merged by the item
that finishes last: the work plan's claim counter and per-query completion counters are
rebuilt inside the graph on every replay, and a replay that reused stale counters would
lose or double items."""
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


def _inputs(synth, nq, N, D, lengths, seed, dev):
    """Queries and CSR lists with the given per-query lengths (ids distinct within a list)."""
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    Q = torch.randn(nq, D, generator=g, device=dev)
    Q = Q / Q.norm(dim=1, keepdim=True)
    off, ids = synth.candidate_lists(nq, N, lengths, g, dev)
    return Q, off, ids


@pytest.mark.parametrize("schedule", [1, 0, 3])
def test_captured_search_replays_match_eager_launches(glv, schedule):
    from paper_2410_22347_gb300 import synth
    dev = torch.device("cuda:0")
    nq, N, D, d, C, kappa, k = 700, 60000, 128, 40, 6, 50, 10
    w = synth.make_workload(N=N, D=D, d=d, C=C, nq=nq, K_db=8, cands=("lognormal", 1500.0, 1.2, 64, 20000),
                            kappa=kappa, k=k, cfg=95, device=dev)
    lengths = (w.off[1:] - w.off[:-1]).clone()
    assert int(lengths.max()) >= 2 * 4096, "the case must contain lists that are cut into work items"
    tags = glv.glv_assign_tags(w.X, w.mu)
    Xred, scales = glv.glv_build_reduced(w.X, tags, w.B, glv.GLV_BF16)
    rs = glv.min_row_stride(d, glv.GLV_BF16)
    n_cand = int(w.off[-1])
    prev = glv.glv_get_score_config(glv.GLV_BF16, d)
    glv.glv_set_score_config(glv.GLV_BF16, 0, 0, 0, schedule)
    try:
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        # captured buffers
        Qs = w.Q.clone()
        offs = w.off.clone()
        idss = w.ids.clone()
        ws = torch.empty(glv._lib.glv_search_workspace_size(nq, D, C, d, glv.GLV_BF16, n_cand, kappa),
                         dtype=torch.uint8, device=dev)
        out_s = torch.empty(nq, k, dtype=torch.float32, device=dev)
        out_id = torch.empty(nq, k, dtype=torch.int32, device=dev)

        def step(stream=None):
            glv.glv_search(w.X, Qs, w.A, glv.GLV_BF16, Xred, rs, scales, glv.GLV_BF16, tags, offs, idss, kappa, k,
                           workspace=ws, out_s=out_s, out_id=out_id, d_status=st, stream=stream)

        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            step()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        torch.cuda.synchronize()

        perm_gen = torch.Generator(device="cpu")
        perm_gen.manual_seed(7)
        for rep in range(3):
            # new queries and new lists with the same total length (a permutation of the lengths)
            L = lengths[torch.randperm(nq, generator=perm_gen).to(dev)] if rep else lengths
            Qn, offn, idsn = _inputs(synth, nq, N, D, L, 1000 + rep, dev)
            assert int(offn[-1]) == n_cand
            Qs.copy_(Qn)
            offs.copy_(offn)
            idss.copy_(idsn)
            graph.replay()
            torch.cuda.synchronize()
            g_s, g_id = out_s.clone(), out_id.clone()
            # eager launches of the same calls on separate buffers
            e_s, e_id = glv.glv_search(w.X, Qn, w.A, glv.GLV_BF16, Xred, rs, scales, glv.GLV_BF16, tags, offn, idsn,
                                       kappa, k, d_status=st)
            torch.cuda.synchronize()
            assert int(st.item()) == 0
            assert torch.equal(g_id, e_id), f"replay {rep}: ids differ from eager launches"
            assert torch.equal(g_s.view(torch.int32), e_s.view(torch.int32)), f"replay {rep}: scores differ"
            assert bool((g_id >= 0).all()), "every query has at least k candidates"
    finally:
        glv.glv_set_score_config(glv.GLV_BF16, prev[0], prev[1], prev[2], prev[3])
