"""Deep zoom (Sec. 3): 64 frames of 1920x1080 centred on seeded points of the
Julia set of C = -0.7269+0.1889i, widths 4 -> 1e-12, limit 2000, precision
chosen per frame by the library (JL_AUTO).  Counts are bit-exact against the
oracle in the precision the library chose (sampled rows of sampled frames, in
the batch launch configuration); the binary32-vs-binary64 mismatch rate is
measured, not pinned."""
import numpy as np
import pytest

import oracle
import paper_1611_03079_b300 as jl
from paper_1611_03079_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def _counts(b, i):
    return b.counts(i).cpu().numpy().view(np.uint16)


def test_deep_zoom_auto_precision_and_parity(cuda):
    import torch
    frames = wl.deep_zoom()
    for f in frames:
        f["rgba"] = False
    b = jl.Batch(frames)
    b.launch()
    torch.cuda.synchronize()
    assert b.status() == 0
    precs = b.precisions()
    assert precs == [oracle.precision_for_view(f["rect"], f["W"], f["H"]) for f in frames]
    n64 = sum(precs)
    assert 50 <= n64 <= 60
    for i in (0, 5, 12, 30, 45, 63):
        f = frames[i]
        rows = [0, 333, 540, 1079]
        k = oracle.render_rows(f["c"], f["rect"], f["W"], f["H"], rows, f["max_iter"], 0, precs[i])
        assert (_counts(b, i)[rows] == k).all(), i
    b.close()


def test_fp32_vs_fp64_mismatch_is_measured(cuda):
    """Forced binary32 and binary64 renders of the same deep-zoom frames are
    each exact against the oracle in their own precision; the fraction of
    pixels where they differ grows with depth."""
    import torch
    frames = wl.deep_zoom()
    pick = [2, 20, 40]
    rates = []
    for i in pick:
        f = dict(frames[i])
        f["W"], f["H"] = 480, 270
        w = f["rect"][1] - f["rect"][0]
        h = w * 270 / 480
        cx, cy = (f["rect"][0] + f["rect"][1]) / 2, (f["rect"][2] + f["rect"][3]) / 2
        f["rect"] = (cx - w / 2, cx + w / 2, cy - h / 2, cy + h / 2)
        out = {}
        for p in (0, 1):
            r = jl.render(f["c"], f["rect"], 480, 270, f["max_iter"], precision=p, count_type="u16", rgba=False)
            torch.cuda.synchronize()
            out[p] = r["counts"].view(torch.int16).cpu().numpy().view(np.uint16)
            assert (out[p] == oracle.render(f["c"], f["rect"], 480, 270, f["max_iter"], 0, p)).all()
        rates.append(float((out[0] != out[1]).mean()))
    assert rates[0] < rates[-1]
    assert rates[-1] > 0.5
