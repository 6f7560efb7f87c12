"""Launch-shape tuning on the GPU: vca_autotune measures the candidate shapes and records the
fastest; every shape (CTA size of the CUDA-core form, CTA count of the tensor-core form) gives the
same features bit for bit; an analyzer opened with VCA_KERNEL_AUTO follows the table; a batch's
tuned SM split keeps its features identical to single analyzers'."""

import pytest

from synth import SequenceSpec, frames_list, tiny_spec
from vca_testutil import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vca():
    import torch

    from paper_2304_12384_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2304_12384_gb300 import vca as v
    yield v
    v.vca_tune_clear()  # the table is process-wide: leave it empty for later tests


def _features(vca, frames, kernel, **kw):
    an = vca.Analyzer(640, 352, 8, 32, kw.pop("low_pass", True), kernel=kernel, max_batch=len(frames))
    try:
        an.push(*to_device(frames))
        return [an.frame_features(t) for t in range(len(frames))], an.kernel
    finally:
        an.close()


def test_autotune_picks_a_measured_candidate_and_shapes_agree(vca):
    import torch

    frames = frames_list(tiny_spec(21))[:6]
    y, u, v = to_device(frames)
    cfg = vca._config(640, 352, 8, 32, True)
    vca.vca_tune_clear()
    chosen, cands = vca.vca_autotune(cfg, y, u, v, reps=3)
    torch.cuda.synchronize()
    kinds = {(c["kernel"], c["plain_warps"], c["tc_ctas"]) for c in cands}
    assert {(1, 2, 0), (1, 4, 0), (1, 8, 0)} <= kinds and any(k[0] == 2 for k in kinds)
    assert all(c["ms_per_frame"] > 0 for c in cands)
    assert chosen["ms_per_frame"] == min(c["ms_per_frame"] for c in cands)
    assert vca.vca_tune_lookup(cfg) == chosen
    # every candidate shape gives the same features, bit for bit, as the default shapes
    ref_plain, _ = _features(vca, frames, vca.VCA_KERNEL_PLAIN)
    ref_tc, _ = _features(vca, frames, vca.VCA_KERNEL_TC)
    for c in cands:
        vca.vca_tune_set(**dict(c))
        got, k = _features(vca, frames, c["kernel"])
        assert k == c["kernel"]
        assert got == (ref_plain if c["kernel"] == 1 else ref_tc), c
    # AUTO follows the table's kernel
    for kern in (1, 2):
        vca.vca_tune_set(**dict(chosen, kernel=kern, plain_warps=2, tc_ctas=6))
        got, k = _features(vca, frames, vca.VCA_KERNEL_AUTO)
        assert k == kern and got == (ref_plain if kern == 1 else ref_tc)
    vca.vca_tune_clear()


def test_batch_split_weight_tuning_keeps_features(vca):
    specs = [SequenceSpec(640, 352, 3, 71, bit_depth=8), SequenceSpec(320, 192, 3, 72, bit_depth=10),
             SequenceSpec(640, 352, 3, 73, bit_depth=10)]
    fr = [frames_list(sp) for sp in specs]
    dev = [to_device(f) for f in fr]
    singles = []
    for sp, d in zip(specs, dev):
        a = vca.Analyzer(sp.width, sp.height, sp.bit_depth, 32, True, max_batch=3)
        a.push(*d)
        singles.append([a.frame_features(t) for t in range(3)])
        a.close()
    ans = [vca.Analyzer(sp.width, sp.height, sp.bit_depth, 32, True, max_batch=1) for sp in specs]
    b = vca.Batch(ans)
    try:
        assert b.kernel == vca.VCA_KERNEL_TC
        refs = [b.frame_refs([(d[0][t], d[1][t], d[2][t]) for d in dev]) for t in range(3)]
        w, ms = b.autotune(refs[0], reps=4)  # 2 warm-up + 4 timed ticks per weight, all of frame 0
        assert any(abs(w - c) < 1e-6 for c in (1.0, 1.15, 1.3, 1.5, 1.75)) and ms > 0
        with pytest.raises(vca.VcaError):
            b.set_split_weight(9.0)
        b.sync()
    finally:  # the tuning ticks advanced the members' h state: compare with fresh analyzers
        b.close()
        for a in ans:
            a.close()
    ans = [vca.Analyzer(sp.width, sp.height, sp.bit_depth, 32, True, max_batch=1) for sp in specs]
    b = vca.Batch(ans)
    try:
        b.set_split_weight(w)
        for t in range(3):
            b.tick([(d[0][t], d[1][t], d[2][t]) for d in dev])
        b.sync()
        for i, a in enumerate(ans):
            assert [a.frame_features(t) for t in range(3)] == singles[i], i
    finally:
        b.close()
        for a in ans:
            a.close()
