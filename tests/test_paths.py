"""Parameter paths of Sec. 3, pinned by the values printed in Fig. 2 and
Fig. 3 (tests/golden/)."""
import math
import os

import numpy as np

from paper_1611_03079_b300 import paths

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    rows = [l.split() for l in open(os.path.join(GOLDEN, name)) if l.strip() and not l.startswith("#")]
    return [complex(float(a), float(b)) for a, b in rows]


def test_fig2_values_lie_on_the_a39_cardioid_clockwise():
    """The four Fig. 2 values lie on f(t) with a = 3.9 to the printed six
    digits, and in caption order t decreases (clockwise)."""
    ts = []
    for c in load("fig2_cardioid_c.txt"):
        t, d = paths.fit_cardioid_parameter(c, 3.9)
        assert d < 1e-6, (c, d)
        # but not on the a = 4 boundary cardioid
        assert paths.fit_cardioid_parameter(c, 4.0)[1] > 1e-3
        ts.append(t)
    # clockwise: each next value is reached by decreasing t (mod 2 pi)
    steps = [((ts[i] - ts[i + 1]) % (2 * math.pi)) for i in range(len(ts) - 1)]
    assert all(0 < s < math.pi for s in steps), ts


def test_cardioid_path_and_sweep():
    a = paths.cardioid_path(720)
    assert abs(a[0] - paths.cardioid_point(0.0)) == 0.0
    # clockwise: the imaginary part decreases right after t = 0
    assert a[1].imag < a[0].imag
    # a = 3.9 keeps C outside the main cardioid: |1 - sqrt(1 - 4c)| > 1
    for c in a[::7]:
        assert abs(1 - np.sqrt(1 - 4 * c)) > 1.0
    s = paths.expanding_sweep(100, 3, 3.9, 3.0)
    assert len(s) == 300
    r = [abs(c - 0.25) for c in s]
    assert r[-1] > r[0]
    assert max(abs(s[i + 1] - s[i]) for i in range(len(s) - 1)) < 0.1


def test_fig3_values_are_close_and_near_the_boundary():
    """Fig. 3's two values are 'very close' (|dC| ~ 0.014) and both sit just
    outside the main cardioid, near the Mandelbrot boundary."""
    c1, c2 = load("fig3_deep_zoom_c.txt")
    assert abs(c1 - c2) < 0.02
    for c in (c1, c2):
        q = abs(1 - np.sqrt(1 - 4 * c))
        assert 1.0 < q < 1.15


def test_frame_builders():
    fr = paths.with_minimap(paths.julia_frames(paths.cardioid_path(4), W=64, H=48))
    assert len(fr) == 8 and fr[1]["mode"] == 1 and fr[0]["mode"] == 0
    z = paths.mandelbrot_zoom(load("fig3_deep_zoom_c.txt")[0], 5)
    w = [f["rect"][1] - f["rect"][0] for f in z]
    assert w[0] == 3.0 and abs(w[-1] - 1e-12) < 1e-15 and all(w[i + 1] < w[i] for i in range(4))
