"""The frame reduction is exact: every feature equals the exact sum of its block values, rounded
once to FP64 and divided by its norm (Section 2 of the paper, the frame features E, h and L).

Block values are synthetic, drawn from the domain the analyzer writes (0, or floats in [1, 2^30):
H is a sum of weights >= 1 times integers, L the square root of an integer), including frames
whose sums pass 2^64 in units of 2^-23.  The expected features come from Python integers: each
value times 2^23 is an integer (its significand shifted by its exponent), the sums are exact,
Python's int-to-float conversion rounds to nearest and its division is IEEE division.  The
features must match bit for bit, whatever the frame size (and so the number of slices).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [  # (blocks per plane C, frames, H exponent range)
    (100, 4, (0, 20)),
    (8160, 3, (0, 27)),
    (40000, 2, (29, 30)),  # H sums beyond 2^64 units of 2^-23
]


@pytest.fixture(scope="module")
def vca():
    import torch

    from paper_2304_12384_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2304_12384_gb300 import vca as v
    return v


def _values(rng, n, erange):
    """n float32 values: a tenth zeros, the rest 2^U(erange) rounded to float32 (below 2^30)."""
    v = np.minimum(np.exp2(rng.uniform(erange[0], erange[1], n)), 2.0 ** 30 - 64).astype(np.float32)
    v[rng.random(n) < 0.1] = 0.0
    return v


def _fixed(v):
    """v * 2^23 as Python integers (v is 0 or a float32 >= 1)."""
    b = v.view(np.uint32).astype(np.int64)
    e = (b >> 23) - 127
    m = (b & 0x7FFFFF) | 0x800000
    q = np.where(b == 0, 0, m << np.maximum(e, 0))
    return [int(x) for x in q]


def _expected(bv, prev, w):
    C = bv.shape[2]
    normY, normC = float(C * w * w), float(C * (w // 2) ** 2)
    out = []
    for t in range(bv.shape[0]):
        rows = [_fixed(bv[t, r]) for r in range(6)]
        tot = [sum(r) for r in rows]
        before = bv[t - 1, 0] if t > 0 else prev
        if before is None:
            dh = 0
        else:
            dh = sum(abs(a - b) for a, b in zip(rows[0], _fixed(before)))
        f = lambda q, norm: float(q) * 2.0 ** -23 / norm  # noqa: E731
        out.append([f(tot[0], normY), f(dh, normY), f(tot[1], C), f(tot[2], normC), f(tot[4], normC),
                    f(tot[3], C), f(tot[5], C)])
    return out


@pytest.mark.parametrize("C,nf,erange", CASES)
def test_features_are_the_exact_sums_rounded_once(vca, C, nf, erange):
    import torch

    rng = np.random.default_rng(C + nf)
    bv = np.stack([np.stack([_values(rng, C, erange if r % 2 == 0 else (0, 12)) for r in range(6)]) for _ in range(nf)])
    prev = _values(rng, C, erange)
    if erange[0] >= 29:
        assert sum(_fixed(bv[0, 0])) >= 2 ** 64  # the case reaches the high word
    exp = _expected(bv, prev, 32)
    bv_dev = torch.from_numpy(bv).cuda()
    prev_dev = torch.from_numpy(prev).cuda()
    last = torch.zeros(C, dtype=torch.float32, device="cuda")
    feats = torch.zeros(nf, 8, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    vca.vca_reduce_frames_noalloc(bv_dev.data_ptr(), C, 32, nf, prev_dev.data_ptr(), last.data_ptr(),
                                  feats.data_ptr(), stream)
    torch.cuda.synchronize()
    got = feats.cpu().numpy()[:, :7].tolist()
    assert got == exp
    assert torch.equal(last, bv_dev[nf - 1, 0])
    # without a previous frame, h of the first frame is 0
    vca.vca_reduce_frames_noalloc(bv_dev.data_ptr(), C, 32, 1, None, last.data_ptr(), feats.data_ptr(), stream)
    torch.cuda.synchronize()
    assert feats[0, 1].item() == 0.0 and feats[0, 0].item() == exp[0][0]
