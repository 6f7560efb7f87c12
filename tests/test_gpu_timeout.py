"""The bounded-wait failure path of the tensor-core kernel, exercised without any fault: the test
hook sets a short wait limit and withholds the copies of one tile, so the convert warps' wait for
that tile runs out.  The push (or batched tick) must report VCA_E_TIMEOUT, the kernel must have
released its tensor memory (later launches on the same SMs run), and the next frames on the same
analyzer (batch) must give the oracle's features, their h chain restarted."""

import pytest

from synth import SequenceSpec, frames_list, tiny_spec
from vca_testutil import assert_features_close, oracle_config, oracle_sequence, to_device

pytestmark = pytest.mark.gpu

LIMIT_NS = 50_000_000  # 50 ms: far above any normal wait of these small launches


@pytest.fixture(scope="module")
def vca():
    import torch

    from paper_2304_12384_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2304_12384_gb300 import vca as v
    return v


@pytest.mark.parametrize("withhold", [0, 3])
def test_single_analyzer_reports_timeout_and_recovers(vca, withhold):
    frames = frames_list(tiny_spec(31))[:12]
    y, u, v = to_device(frames)
    an = vca.Analyzer(640, 352, 8, 32, True, kernel=vca.VCA_KERNEL_TC, max_batch=4)
    try:
        an.push(y[0:4], u[0:4], v[0:4])
        for t in range(4):
            an.frame_features(t)
        vca.vca_debug_wait(an.handle, LIMIT_NS, withhold)
        an.push(y[4:8], u[4:8], v[4:8])
        for lost in (4, 7):  # every frame of the push is lost, and says so
            with pytest.raises(vca.VcaError) as ei:
                an.frame_features(lost)
            assert ei.value.status == vca.VCA_E_TIMEOUT
        # recovery on the same analyzer (the limit stays short, nothing is withheld any more)
        an.push(y[8:12], u[8:12], v[8:12])
        per, _ = oracle_sequence(frames[8:12], oracle_config(an))  # h restarts at frame 8
        for t in range(4):
            assert_features_close(an.frame_features(8 + t), per[t], where=f"frame {8 + t}")
        vca.vca_debug_wait(an.handle, 0, -1)
    finally:
        an.close()
    # a fresh analyzer on the same device runs too
    an = vca.Analyzer(640, 352, 8, 32, True, kernel=vca.VCA_KERNEL_TC, max_batch=4)
    try:
        an.push(y[0:4], u[0:4], v[0:4])
        per, _ = oracle_sequence(frames[0:4], oracle_config(an))
        assert_features_close(an.frame_features(3), per[3], where="fresh analyzer")
    finally:
        an.close()


def test_batched_tick_reports_timeout_and_recovers(vca):
    specs = [SequenceSpec(640, 352, 6, 81, bit_depth=8), SequenceSpec(320, 192, 6, 82, bit_depth=10)]
    fr = [frames_list(sp) for sp in specs]
    dev = [to_device(f) for f in fr]
    ans = [vca.Analyzer(sp.width, sp.height, sp.bit_depth, 32, True, max_batch=1) for sp in specs]
    b = vca.Batch(ans)
    try:
        assert b.kernel == vca.VCA_KERNEL_TC
        b.tick([(d[0][0], d[1][0], d[2][0]) for d in dev])
        b.sync()
        vca.vca_batch_debug_wait(b.handle, LIMIT_NS, 1)
        b.tick([(d[0][1], d[1][1], d[2][1]) for d in dev])
        with pytest.raises(vca.VcaError) as ei:
            b.sync()
        assert ei.value.status == vca.VCA_E_TIMEOUT
        for t in range(2, 6):
            b.tick([(d[0][t], d[1][t], d[2][t]) for d in dev])
        b.sync()
        for i, a in enumerate(ans):
            with pytest.raises(vca.VcaError) as ei:
                a.frame_features(1)
            assert ei.value.status == vca.VCA_E_TIMEOUT
            per, _ = oracle_sequence(fr[i][2:6], oracle_config(a))  # h restarts at frame 2
            for t in range(4):
                assert_features_close(a.frame_features(2 + t), per[t], where=f"member {i} frame {2 + t}")
    finally:
        b.close()
        for a in ans:
            a.close()


def test_hook_rules(vca):
    an = vca.Analyzer(640, 352, 8, 32, True, kernel=vca.VCA_KERNEL_PLAIN, max_batch=1)
    try:
        with pytest.raises(vca.VcaError) as ei:
            vca.vca_debug_wait(an.handle, LIMIT_NS, 0)
        assert ei.value.status == vca.VCA_E_UNSUPPORTED
    finally:
        an.close()
    an = vca.Analyzer(640, 352, 8, 32, True, kernel=vca.VCA_KERNEL_TC, max_batch=1)
    try:
        with pytest.raises(vca.VcaError) as ei:
            vca.vca_debug_wait(an.handle, -1, 0)
        assert ei.value.status == vca.VCA_E_ARG
    finally:
        an.close()
