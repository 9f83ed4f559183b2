"""Learned screening surrogate: Python binding of the jl_model_* / jl_train /
jl_survey / jl_topk entry points, plus the screening workflow built from
library calls only (argument marshalling; every numeric step runs in the
library's kernels).

Workflow (the paper's aim of sampling the parameter space quickly, Sec. 1,
with the Mandelbrot set as the roadmap for C, Sec. 3):
  1. render the escape-count histograms of training values of C with a batch
     plan (one CUDA-graph launch), the targets;
  2. train the network on the device (tcgen05 forward and backward, Adam);
  3. screen many candidate C by predicted histogram: score = entropy of the
     prediction, keep the top k;
  4. judge: render the kept C for real and measure the histogram L1 distance
     between prediction and rendering.
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import check

N_BINS = 101
SURVEY_RECT = (-2.0, 2.0, -2.0, 2.0)
SURVEY_W = SURVEY_H = 128
SURVEY_MAX_ITER = 100

# numpy mirror of jl_frame (include/jl.h): 96 bytes, natural alignment
FRAME_DTYPE = np.dtype([("cr", "f8"), ("ci", "f8"), ("xmin", "f8"), ("xmax", "f8"), ("ymin", "f8"),
                        ("ymax", "f8"), ("width", "i4"), ("height", "i4"), ("max_iter", "i4"), ("mode", "i4"),
                        ("precision", "i4"), ("count_type", "i4"), ("counts_offset", "i8"),
                        ("rgba_offset", "i8"), ("hist_offset", "i8")])
assert FRAME_DTYPE.itemsize == ctypes.sizeof(_lib.Frame)


class HistogramPlan:
    """Batch plan rendering only the normalised histograms of Julia frames
    (128x128 over [-2,2]^2, limit 100 by default) for an array of C."""

    def __init__(self, c, rect=SURVEY_RECT, W=SURVEY_W, H=SURVEY_H, max_iter=SURVEY_MAX_ITER, precision=0,
                 chunk_len=0):
        import torch
        c = np.asarray(c, dtype=np.float64).reshape(-1, 2)
        n = c.shape[0]
        self.n, self.bins = n, int(max_iter) + 1
        fr = np.zeros(n, dtype=FRAME_DTYPE)
        fr["cr"], fr["ci"] = c[:, 0], c[:, 1]
        fr["xmin"], fr["xmax"], fr["ymin"], fr["ymax"] = rect
        fr["width"], fr["height"], fr["max_iter"] = W, H, max_iter
        fr["mode"], fr["precision"], fr["count_type"] = 0, precision, 0
        fr["counts_offset"], fr["rgba_offset"] = -1, -1
        fr["hist_offset"] = np.arange(n, dtype=np.int64) * self.bins * 4
        self.hist = torch.empty((n, self.bins), dtype=torch.float32, device="cuda")
        self._L = _lib.lib()
        opts = _lib.BatchOpts()
        opts.chunk_len = int(chunk_len)
        h = ctypes.c_void_p()
        check(self._L.jl_batch_create(fr.ctypes.data, n, None, None, self.hist.data_ptr(), None, ctypes.byref(opts),
                                      ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        import torch
        st = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        check(self._L.jl_batch_launch(self._h, st))
        return self.hist

    def close(self):
        if getattr(self, "_h", None):
            self._L.jl_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def render_histograms(c, **kw):
    """Histograms (torch, n x (max_iter+1), device) of the Julia frames of c."""
    import torch
    p = HistogramPlan(c, **kw)
    h = p.launch()
    torch.cuda.synchronize()
    p.close()
    return h


def hist_l1(p, q):
    """Per-row L1 distance of two (n x b) device histogram tensors."""
    import torch
    n, b = p.shape
    out = torch.empty(n, dtype=torch.float32, device=p.device)
    st = torch.cuda.current_stream().cuda_stream
    check(_lib.lib().jl_hist_l1(p.data_ptr(), p.stride(0), q.data_ptr(), q.stride(0), n, b, out.data_ptr(), st))
    return out


def topk(score, k):
    """(indices, scores) of the k largest scores, ties by smaller index."""
    import torch
    n = score.numel()
    idx = torch.empty(k, dtype=torch.int32, device=score.device)
    val = torch.empty(k, dtype=torch.float32, device=score.device)
    st = torch.cuda.current_stream().cuda_stream
    check(_lib.lib().jl_topk(score.data_ptr(), n, int(k), idx.data_ptr(), val.data_ptr(), st))
    return idx, val


PARAM_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


class Surrogate:
    """The surrogate network on the current device (jl_model)."""

    def __init__(self, fourier_B, init_params):
        self._L = _lib.lib()
        B = np.ascontiguousarray(fourier_B, dtype=np.float32).reshape(32, 2)
        flat = np.concatenate([np.asarray(init_params[k], np.float32).ravel() for k in PARAM_ORDER])
        if flat.size != self._L.jl_model_num_params():
            raise ValueError("parameter block has %d values, expected %d" % (flat.size,
                                                                             self._L.jl_model_num_params()))
        h = ctypes.c_void_p()
        check(self._L.jl_model_create(B.ctypes.data, flat.ctypes.data, ctypes.byref(h)))
        self._h = h

    @classmethod
    def load(cls, path):
        self = cls.__new__(cls)
        self._L = _lib.lib()
        h = ctypes.c_void_p()
        check(self._L.jl_model_load(str(path).encode(), ctypes.byref(h)))
        self._h = h
        return self

    def save(self, path):
        check(self._L.jl_model_save(self._h, str(path).encode()))

    def state(self):
        n = self._L.jl_model_num_params()
        p, m, v = (np.zeros(n, np.float32) for _ in range(3))
        s = ctypes.c_int32(0)
        check(self._L.jl_model_get_state(self._h, p.ctypes.data, m.ctypes.data, v.ctypes.data, ctypes.byref(s)))
        return p, m, v, s.value

    def forward(self, c, probs=True, score=True):
        """c: torch (n, 2) float32 on the device.  Returns (probs, score)."""
        import torch
        n = c.shape[0]
        P = torch.empty((n, N_BINS), dtype=torch.float32, device=c.device) if probs else None
        S = torch.empty(n, dtype=torch.float32, device=c.device) if score else None
        st = torch.cuda.current_stream().cuda_stream
        check(self._L.jl_model_forward(self._h, c.data_ptr(), n, P.data_ptr() if probs else None,
                                       S.data_ptr() if score else None, st))
        return P, S

    @staticmethod
    def epoch_order(n, epochs, order_seed=0):
        """The sample order train() uses: one seeded permutation of n samples
        per epoch (host int32 array, epochs * n)."""
        rng = np.random.default_rng(order_seed)
        return np.concatenate([rng.permutation(n).astype(np.int32) for _ in range(epochs)])

    def train(self, c, hist, epochs, batch=1024, lr=1e-3, lr_final=None, order_seed=0, loss_curve=True, order=None):
        """Adam training with a cosine learning-rate schedule from lr to
        lr_final (default: constant lr); one seeded permutation of the
        samples per epoch (epoch_order, drawn on the host), or `order`: those
        permutations already on the device (int32, epochs * n)."""
        import torch
        n = c.shape[0]
        if order is None:
            od = torch.from_numpy(self.epoch_order(n, epochs, order_seed)).to(c.device)
        else:
            od = order
            assert od.dtype == torch.int32 and od.numel() == epochs * n and od.device == c.device
        curve = np.zeros(epochs, np.float32)
        st = torch.cuda.current_stream().cuda_stream
        check(self._L.jl_train(self._h, c.data_ptr(), hist.data_ptr(), n, od.data_ptr(), int(epochs), int(batch),
                               ctypes.c_float(lr), ctypes.c_float(lr if lr_final is None else lr_final),
                               curve.ctypes.data if loss_curve else None, st))
        return curve

    def survey(self, c, k, out=None):
        """Screen c (torch n x 2): returns (top_idx, top_score, score).  `out`
        may supply (top_idx int32[k], top_score float32[k], score float32[n]);
        repeated calls with the same c and outputs replay one CUDA graph."""
        import torch
        n = c.shape[0]
        if out is not None:
            idx, val, S = out
        else:
            S = torch.empty(n, dtype=torch.float32, device=c.device)
            idx = torch.empty(int(k), dtype=torch.int32, device=c.device)
            val = torch.empty(int(k), dtype=torch.float32, device=c.device)
        st = torch.cuda.current_stream().cuda_stream
        check(self._L.jl_survey(self._h, c.data_ptr(), n, int(k), idx.data_ptr(), val.data_ptr(), S.data_ptr(), st))
        return idx, val, S

    def close(self):
        if getattr(self, "_h", None):
            self._L.jl_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
