"""Host checks of the scoring-configuration space the autotuner searches (no GPU): capped
shared-memory carveouts only, the 512-thread schedules only where they are instantiated, and
every schedule bit (planned items, wide CTAs, L2 prefetch) reachable and kept through the
library's resolution of a configuration."""
import pytest


@pytest.fixture(scope="module")
def glv():
    from paper_2410_22347_gb300 import build_lib
    build_lib.build()
    from paper_2410_22347_gb300 import glv as g
    return g


@pytest.mark.parametrize("dt_name", ["f32", "bf16", "fp8"])
def test_configuration_space(glv, dt_name):
    from paper_2410_22347_gb300.autotune import configurations
    dt = glv.DTYPES[dt_name]
    cfgs = list(configurations(dt))
    assert len(cfgs) == len(set(cfgs))
    assert {c for _, _, c, _ in cfgs} == {132, 164}  # the driver's choice (0) is not offered
    smaller = set(glv.SCORE_GROUPS[dt][:2])
    for G, mode, _, sched in cfgs:
        if sched & 2:  # wide CTAs exist for register loads and the two smaller lane counts only
            assert mode == 0 and G in smaller
    assert {s for _, _, _, s in cfgs} == set(range(8))


def test_schedule_bits_survive_resolution(glv):
    dt = glv.GLV_BF16
    try:
        glv.glv_set_score_config(dt, 4, 0, 164, 5)   # planned items + prefetch
        assert glv.glv_get_score_config(dt, 160)[3] == 5
        glv.glv_set_score_config(dt, 16, 0, 164, 7)  # no wide kernel with 16 lanes: bit 1 dropped
        assert glv.glv_get_score_config(dt, 160)[3] == 5
        glv.glv_set_score_config(dt, 8, 1, 0, 6)     # nor with pipelined loads
        assert glv.glv_get_score_config(dt, 160)[3] == 4
    finally:
        glv.glv_set_score_config(dt, 0, 0)
