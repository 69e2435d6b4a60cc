"""CPU oracle for the nucleus pipeline (TEST INFRASTRUCTURE ONLY).

Plain single-threaded C (``oracle.c``) written from the definitions of each
step (Sec. II / Fig. 1 and Table I of Teodoro et al.), FP64 for features.  It
shares no code with the CUDA path.  Only the tests, ``__graft_entry__.smoke``
and the benchmark's CPU-baseline leg may import this package; the library
never does.
"""
import ctypes
import os
import subprocess

import numpy as np

_here = os.path.dirname(os.path.abspath(__file__))
_lib = None
NFEAT = 15
CANNY_LOW, CANNY_HIGH = 40, 120   # hysteresis thresholds on the L1 Sobel magnitude of hem8 (our reading)
EDGE_R = 3                        # radius of the disk dilation the edge counts cover (our reading)
RBC_LO, RBC_HI = 40, 100          # red-dominance thresholds of the RBC mask and markers (our reading)

u8p = ctypes.POINTER(ctypes.c_uint8)
i32p = ctypes.POINTER(ctypes.c_int32)


class ReconStats(ctypes.Structure):
    _fields_ = [("fifo_pushes", ctypes.c_longlong), ("max_depth", ctypes.c_int)]


def build(force=False):
    """Compile liboracle.so next to this file (plain gcc -O2, no OpenMP)."""
    so = os.path.join(_here, "liboracle.so")
    src = os.path.join(_here, "oracle.c")
    hdr = os.path.join(_here, "oracle.h")
    stale = (not os.path.exists(so) or os.path.getmtime(so) < max(os.path.getmtime(src),
                                                                  os.path.getmtime(hdr)))
    if force or stale:
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", so, src, "-lm"])
    return so


def _load():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, ci, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        L.oracle_deconv_tables.argtypes = [vp, vp, vp]
        L.oracle_deconv.argtypes = [vp, ci, ci, sz, vp]
        L.oracle_recon.argtypes = [vp, vp, ci, ci, vp, vp]
        L.oracle_recon.restype = ci
        L.oracle_recon_plain.argtypes = [vp, vp, ci, ci, vp]
        L.oracle_recon_plain.restype = ci
        L.oracle_recon_rounds.argtypes = [vp, vp, ci, ci, vp, vp]
        L.oracle_recon_rounds.restype = ci
        L.oracle_hdome.argtypes = [vp, ci, ci, ci, ci, vp, vp, vp]
        L.oracle_fill_holes.argtypes = [vp, ci, ci, vp]
        L.oracle_label.argtypes = [vp, ci, ci, ci, ci, vp]
        L.oracle_label.restype = ci
        L.oracle_edt.argtypes = [vp, ci, ci, vp]
        L.oracle_features.argtypes = [vp, vp, ci, ci, ci, vp]
        L.oracle_seg.argtypes = [vp, ci, ci, sz, ci, ci, ci, ci, vp, vp, vp, vp, vp, vp]
        L.oracle_seg.restype = ci
        L.oracle_morph_disk.argtypes = [vp, ci, ci, ci, ci, vp]
        L.oracle_morph_open.argtypes = [vp, ci, ci, ci, vp]
        L.oracle_morph_open.restype = ci
        L.oracle_watershed.argtypes = [vp, vp, ci, ci, ci, vp]
        L.oracle_watershed.restype = ci
        L.oracle_canny.argtypes = [vp, ci, ci, ci, ci, vp, vp, vp]
        L.oracle_canny.restype = ctypes.c_longlong
        L.oracle_rbc.argtypes = [vp, ci, ci, sz, ci, ci, vp, vp]
        L.oracle_rbc.restype = ctypes.c_longlong
        L.oracle_edge_counts.argtypes = [vp, vp, ci, ci, ci, ci, vp]
        L.oracle_edge_counts.restype = None
        _lib = L
    return _lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def deconv_tables():
    lut = np.zeros(256, np.int32)
    wq = np.zeros(3, np.int32)
    w = np.zeros(3, np.float64)
    _load().oracle_deconv_tables(lut.ctypes.data, wq.ctypes.data, w.ctypes.data)
    return lut, wq, w


def deconv(rgb):
    rgb, p = _c(rgb, np.uint8)
    H, W = rgb.shape[:2]
    out = np.empty((H, W), np.uint8)
    _load().oracle_deconv(p, W, H, W * 3, out.ctypes.data)
    return out


def recon(marker, mask, stats=False):
    marker, pm = _c(marker, np.uint8)
    mask, pk = _c(mask, np.uint8)
    H, W = mask.shape
    out = np.empty((H, W), np.uint8)
    st = ReconStats()
    rc = _load().oracle_recon(pm, pk, W, H, out.ctypes.data, ctypes.addressof(st) if stats else None)
    if rc != 0:
        raise ValueError("marker must not exceed mask")
    return (out, (st.fifo_pushes, st.max_depth)) if stats else out


def recon_plain(marker, mask):
    marker, pm = _c(marker, np.uint8)
    mask, pk = _c(mask, np.uint8)
    H, W = mask.shape
    out = np.empty((H, W), np.uint8)
    it = _load().oracle_recon_plain(pm, pk, W, H, out.ctypes.data)
    return out, it


def recon_rounds(marker, mask):
    """The plain iteration evaluated only where it can change; returns
    (R, steps, pixel evaluations).  steps is the front distance in
    8-connected steps."""
    marker, pm = _c(marker, np.uint8)
    mask, pk = _c(mask, np.uint8)
    H, W = mask.shape
    out = np.empty((H, W), np.uint8)
    ev = ctypes.c_longlong(0)
    it = _load().oracle_recon_rounds(pm, pk, W, H, out.ctypes.data, ctypes.addressof(ev))
    return out, it, ev.value


def hdome(hem8, h=20, thr=10):
    hem8, p = _c(hem8, np.uint8)
    H, W = hem8.shape
    R = np.empty((H, W), np.uint8)
    fg = np.empty((H, W), np.uint8)
    _load().oracle_hdome(p, W, H, h, thr, R.ctypes.data, fg.ctypes.data, None)
    return R, fg


def fill_holes(fg):
    fg, p = _c(fg, np.uint8)
    H, W = fg.shape
    out = np.empty((H, W), np.uint8)
    _load().oracle_fill_holes(p, W, H, out.ctypes.data)
    return out


def label(filled, amin=20, amax=1500):
    filled, p = _c(filled, np.uint8)
    H, W = filled.shape
    out = np.empty((H, W), np.int32)
    K = _load().oracle_label(p, W, H, amin, amax, out.ctypes.data)
    return out, K


def edt(labels):
    labels, p = _c(labels, np.int32)
    H, W = labels.shape
    out = np.empty((H, W), np.int32)
    _load().oracle_edt(p, W, H, out.ctypes.data)
    return out


def features(hem8, labels, K):
    hem8, ph = _c(hem8, np.uint8)
    labels, pl = _c(labels, np.int32)
    H, W = labels.shape
    out = np.zeros((max(K, 0), NFEAT), np.float64)
    if K > 0:
        _load().oracle_features(ph, pl, W, H, K, out.ctypes.data)
    return out


def seg(rgb, h=20, thr=10, amin=20, amax=1500, planes=False):
    """Run the whole segmentation.  Returns dict with hem8, labels, edt, K
    (and R, fg, filled when planes=True)."""
    rgb, p = _c(rgb, np.uint8)
    H, W = rgb.shape[:2]
    hem8 = np.empty((H, W), np.uint8)
    labels = np.empty((H, W), np.int32)
    ed = np.empty((H, W), np.int32)
    R = np.empty((H, W), np.uint8) if planes else None
    fg = np.empty((H, W), np.uint8) if planes else None
    fl = np.empty((H, W), np.uint8) if planes else None
    ptr = lambda a: a.ctypes.data if a is not None else None
    K = _load().oracle_seg(p, W, H, W * 3, h, thr, amin, amax, hem8.ctypes.data, ptr(R), ptr(fg),
                           ptr(fl), labels.ctypes.data, ed.ctypes.data)
    out = dict(hem8=hem8, labels=labels, edt=ed, K=K)
    if planes:
        out.update(R=R, fg=fg, filled=fl)
    return out


def morph_erode(src, r=9):
    """Grayscale erosion by the disk dx^2 + dy^2 <= r^2 over in-image pixels."""
    src, p = _c(src, np.uint8)
    H, W = src.shape
    out = np.empty((H, W), np.uint8)
    _load().oracle_morph_disk(p, W, H, r, 0, out.ctypes.data)
    return out


def morph_dilate(src, r=9):
    """Grayscale dilation by the same disk."""
    src, p = _c(src, np.uint8)
    H, W = src.shape
    out = np.empty((H, W), np.uint8)
    _load().oracle_morph_disk(p, W, H, r, 1, out.ctypes.data)
    return out


def morph_open(src, r=9):
    """Opening by the disk (Table I "Morph. Open"; r = 9 is the 19 x 19 disk)."""
    src, p = _c(src, np.uint8)
    H, W = src.shape
    out = np.empty((H, W), np.uint8)
    if _load().oracle_morph_open(p, W, H, r, out.ctypes.data) != 0:
        raise ValueError("bad arguments")
    return out


def watershed(labels, edt, h=1):
    """Watershed split of labelled objects on the distance transform (Table I
    "Pre-Watershed" + "Watershed"); returns (split labels, number of basins)."""
    labels, pl = _c(labels, np.int32)
    edt, pe = _c(edt, np.int32)
    H, W = labels.shape
    out = np.empty((H, W), np.int32)
    n = _load().oracle_watershed(pl, pe, W, H, h, out.ctypes.data)
    if n < 0:
        raise ValueError("bad arguments")
    return out, n


def canny(img, low=CANNY_LOW, high=CANNY_HIGH, detail=False):
    """Canny edge map (Sec. V-A feature-stage transform; Table I "Features
    comp."): uint8 plane of 0/1.  detail=True also returns the L1 Sobel
    magnitude and the class plane (0, 1 candidate, 2 strong)."""
    img, p = _c(img, np.uint8)
    H, W = img.shape
    out = np.empty((H, W), np.uint8)
    mag = np.empty((H, W), np.int32)
    cls = np.empty((H, W), np.uint8)
    n = _load().oracle_canny(p, W, H, int(low), int(high), out.ctypes.data, mag.ctypes.data, cls.ctypes.data)
    if n < 0:
        raise ValueError("bad arguments")
    return (out, mag, cls) if detail else out


def edge_counts(edges, labels, K, r=EDGE_R):
    """Edge pixels within each object's disk dilation of radius r (Sec. II
    "edge" features): int32 [K]."""
    edges, pe = _c(edges, np.uint8)
    labels, pl = _c(labels, np.int32)
    H, W = labels.shape
    cnt = np.zeros(max(K, 1), np.int32)
    _load().oracle_edge_counts(pe, pl, W, H, int(K), int(r), cnt.ctypes.data)
    return cnt[:K]


def rbc(rgb, t_lo=RBC_LO, t_hi=RBC_HI, detail=False):
    """Red blood cell mask (Table I "RBC detection"): uint8 plane of 0/1,
    the 8-connected components of {R - max(G, B) >= t_lo} that hold a pixel
    with R - max(G, B) >= t_hi.  detail=True also returns the int16 red
    dominance plane."""
    a = np.asarray(rgb, dtype=np.uint8)
    if a.ndim != 3 or a.shape[2] != 3 or a.strides[1:] != (3, 1):
        a = np.ascontiguousarray(a)
    H, W = a.shape[:2]
    out = np.empty((H, W), np.uint8)
    red = np.empty((H, W), np.int16)
    n = _load().oracle_rbc(a.ctypes.data, W, H, a.strides[0], int(t_lo), int(t_hi), out.ctypes.data,
                           red.ctypes.data)
    if n < 0:
        raise ValueError("bad arguments")
    return (out, red) if detail else out
