"""GB300 per-tile nucleus segmentation + per-object features.

Thin ctypes binding over libpipe.so (C ABI in include/pipe.h).  The names
mirror the C entry points; this module only marshals arguments -- every step
of the path runs in the library's CUDA kernels.  PyTorch tensors serve as
device buffers and torch streams as CUDA streams.  If the library is missing
or fails to load, every call raises: there is no CPU fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpipe.so")
NFEAT = 15

PIPE_OK, PIPE_EINVAL, PIPE_ENOMEM, PIPE_EBUSY, PIPE_EAGAIN, PIPE_ETIMEOUT, PIPE_EOVERFLOW, PIPE_ECUDA = range(8)
STATUS_NAMES = ["PIPE_OK", "PIPE_EINVAL", "PIPE_ENOMEM", "PIPE_EBUSY", "PIPE_EAGAIN", "PIPE_ETIMEOUT",
                "PIPE_EOVERFLOW", "PIPE_ECUDA"]

EXPORTS = ["pipe_default_params", "pipe_create", "pipe_destroy", "seg_tile", "features_tile",
           "seg_features_batch", "batch_submit", "batch_poll", "batch_release", "pipe_serve_memory",
           "pipe_status_read", "pipe_debug_plane",
           "pipe_profile_enable", "pipe_profile_read", "pipe_launch_count", "pipe_recon_visits",
           "features_tile_noalloc", "pipe_autotune_info", "morph_open_tile", "watershed_tile", "canny_tile", "rbc_tile",
           "watershed_batch", "canny_batch", "sched_create", "sched_destroy", "sched_push", "sched_request", "sched_done",
           "sched_release", "sched_counts", "tile_cost"]
NOALLOC_MAX_OBJECTS = 65536


class PipeError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        name = STATUS_NAMES[code] if 0 <= code < len(STATUS_NAMES) else str(code)
        super().__init__("%s failed: %s" % (what, name))


class PipeParams(ctypes.Structure):
    _fields_ = [("h", ctypes.c_int), ("dome_thresh", ctypes.c_int), ("area_min", ctypes.c_int),
                ("area_max", ctypes.c_int), ("glcm_levels", ctypes.c_int), ("n_offsets", ctypes.c_int),
                ("offsets", (ctypes.c_int * 2) * 4), ("hbm_budget_bytes", ctypes.c_size_t),
                ("max_slots", ctypes.c_int), ("wait_budget_cycles", ctypes.c_longlong),
                ("autotune_cache", ctypes.c_char_p), ("autotune", ctypes.c_int)]


class TileDevC(ctypes.Structure):
    _fields_ = [("rgb", ctypes.c_void_p), ("W", ctypes.c_int), ("H", ctypes.c_int),
                ("pitch", ctypes.c_size_t), ("hem8", ctypes.c_void_p), ("labels", ctypes.c_void_p),
                ("edt", ctypes.c_void_p), ("n_objects", ctypes.c_void_p), ("feats", ctypes.c_void_p),
                ("feats_cap", ctypes.c_int)]


class TileDesc(ctypes.Structure):
    _fields_ = [("rgb_host", ctypes.c_void_p), ("W", ctypes.c_int), ("H", ctypes.c_int),
                ("pitch", ctypes.c_size_t), ("want_planes", ctypes.c_int)]


class TileResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("n_objects", ctypes.c_int), ("n_feats", ctypes.c_int),
                ("feats", ctypes.POINTER(ctypes.c_float)), ("hem8", ctypes.POINTER(ctypes.c_uint8)),
                ("labels", ctypes.POINTER(ctypes.c_int32)), ("edt", ctypes.POINTER(ctypes.c_int32)),
                ("t_arrive_ms", ctypes.c_double), ("t_done_ms", ctypes.c_double)]


_lib = None


def lib():
    """Load libpipe.so (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libpipe.so not built (%s); run paper_1209_3332_gb300.build.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, ci, sz, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_uint64
    L.pipe_default_params.argtypes = [ctypes.POINTER(PipeParams)]
    L.pipe_default_params.restype = None
    L.pipe_create.argtypes = [ctypes.POINTER(PipeParams), ci, ctypes.POINTER(vp)]
    L.pipe_destroy.argtypes = [vp]
    L.pipe_destroy.restype = None
    L.seg_tile.argtypes = [vp, vp, ci, ci, sz, vp, vp, vp, vp, vp]
    L.features_tile.argtypes = [vp, vp, vp, ci, ci, ci, vp, vp]
    L.seg_features_batch.argtypes = [vp, ctypes.POINTER(TileDevC), ci, vp]
    L.morph_open_tile.argtypes = [vp, vp, ci, ci, ci, vp, vp]
    L.watershed_tile.argtypes = [vp, vp, vp, ci, ci, ci, ci, vp, vp, vp]
    L.canny_tile.argtypes = [vp, vp, vp, ci, ci, ci, ci, ci, ci, vp, vp, vp]
    L.rbc_tile.argtypes = [vp, vp, ci, ci, sz, ci, ci, vp, vp]
    L.canny_batch.argtypes = [vp, ctypes.POINTER(EdgeTileC), ci, ci, ci, ci, vp]
    L.watershed_batch.argtypes = [vp, ctypes.POINTER(WsTileC), ci, ci, vp]
    L.sched_create.argtypes = [ci, ci, ctypes.POINTER(vp)]
    L.sched_create.restype = ci
    L.sched_destroy.argtypes = [vp]
    L.sched_destroy.restype = None
    L.sched_push.argtypes = [vp, u64, ctypes.c_double]
    L.sched_push.restype = ci
    L.sched_request.argtypes = [vp, ci, ctypes.POINTER(u64)]
    L.sched_request.restype = ci
    L.sched_done.argtypes = [vp, ci, u64]
    L.sched_done.restype = ci
    L.sched_release.argtypes = [vp, ci, ctypes.POINTER(ctypes.c_longlong)]
    L.sched_release.restype = ci
    L.sched_counts.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                               ctypes.POINTER(ctypes.c_longlong)]
    L.sched_counts.restype = ci
    L.tile_cost.argtypes = [vp, ci, ci, sz]
    L.tile_cost.restype = ctypes.c_double
    L.batch_submit.argtypes = [vp, ctypes.POINTER(TileDesc), ci, ctypes.POINTER(u64)]
    L.batch_poll.argtypes = [vp, u64, ctypes.POINTER(ci), ctypes.POINTER(TileResult)]
    L.batch_release.argtypes = [vp, u64]
    L.pipe_serve_memory.argtypes = [vp, ctypes.POINTER(sz), ctypes.POINTER(sz), ctypes.POINTER(ci)]
    L.pipe_status_read.argtypes = [vp]
    L.pipe_debug_plane.argtypes = [vp, ci, vp, vp]
    L.pipe_profile_enable.argtypes = [vp, ci]
    L.pipe_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_longlong),
                                    ctypes.POINTER(ctypes.c_double), ci]
    L.pipe_launch_count.argtypes = [vp]
    L.pipe_launch_count.restype = ctypes.c_longlong
    L.features_tile_noalloc.argtypes = [vp, vp, ci, ci, ci, vp, vp]
    L.features_tile_noalloc.restype = ci
    L.pipe_recon_visits.argtypes = [vp]
    L.pipe_recon_visits.restype = ctypes.c_longlong
    L.pipe_autotune_info.argtypes = [vp, ctypes.POINTER(ci), ctypes.POINTER(ci), ctypes.POINTER(ci),
                                     ctypes.POINTER(ctypes.c_longlong)]
    for n in ("pipe_create", "seg_tile", "features_tile", "seg_features_batch", "batch_submit", "batch_poll",
              "batch_release", "pipe_serve_memory",
              "pipe_status_read", "pipe_debug_plane", "pipe_profile_enable", "pipe_profile_read",
              "morph_open_tile", "watershed_tile", "canny_tile", "watershed_batch", "rbc_tile", "canny_batch"):
        getattr(L, n).restype = ci
    _lib = L
    return L


def _check(rc, what):
    if rc != PIPE_OK:
        raise PipeError(rc, what)


def features_tile_noalloc(hem8, labels, n_objects, feats, stream=None):
    """features_tile on the current device with no allocation (static scratch)."""
    H, W = labels.shape
    rc = lib().features_tile_noalloc(hem8.data_ptr(), labels.data_ptr(), W, H, int(n_objects),
                                     feats.data_ptr() if feats is not None else None, _stream_ptr(stream))
    _check(rc, "features_tile_noalloc")


def default_params():
    p = PipeParams()
    lib().pipe_default_params(ctypes.byref(p))
    return p


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def tile_cost(rgb):
    """Cost estimate of a host RGB tile (H, W, 3) uint8 for the dispatch
    queue: W * H * (1 + 8 * dark fraction on a 1-in-64 sample)."""
    import numpy as np
    a = np.asarray(rgb, dtype=np.uint8)
    if a.ndim != 3 or a.shape[2] != 3 or a.strides[1:] != (3, 1):
        a = np.ascontiguousarray(a)               # rows of packed RGB; a row pitch is kept as it is
    H, W = a.shape[:2]
    c = lib().tile_cost(a.ctypes.data, W, H, a.strides[0])
    if c < 0:
        raise ValueError("bad tile")
    return c


class Sched:
    """Demand-driven dispatch queue (sched_t): workers request tasks, at most
    `window` held each, most expensive first (the paper's Manager window,
    Sec. III-B, with the PATS sorted queue, Sec. IV-B)."""

    def __init__(self, n_workers, window):
        h = ctypes.c_void_p()
        _check(lib().sched_create(int(n_workers), int(window), ctypes.byref(h)), "sched_create")
        self.h = h

    def push(self, task, cost):
        _check(lib().sched_push(self.h, int(task), float(cost)), "sched_push")

    def request(self, worker):
        """The granted task id, or None when nothing is queued; raises
        PipeError(PIPE_EBUSY) when the worker's window is full."""
        t = ctypes.c_uint64()
        rc = lib().sched_request(self.h, int(worker), ctypes.byref(t))
        if rc == PIPE_EAGAIN:
            return None
        _check(rc, "sched_request")
        return t.value

    def done(self, worker, task):
        _check(lib().sched_done(self.h, int(worker), int(task)), "sched_done")

    def release(self, worker):
        """Return every task the worker holds to the queue (failure
        recovery); the number returned."""
        n = ctypes.c_longlong()
        _check(lib().sched_release(self.h, int(worker), ctypes.byref(n)), "sched_release")
        return n.value

    def counts(self):
        q, f, c = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(lib().sched_counts(self.h, ctypes.byref(q), ctypes.byref(f), ctypes.byref(c)), "sched_counts")
        return q.value, f.value, c.value

    def close(self):
        if self.h:
            lib().sched_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class EdgeTileC(ctypes.Structure):
    _fields_ = [("img", ctypes.c_void_p), ("labels", ctypes.c_void_p), ("W", ctypes.c_int), ("H", ctypes.c_int),
                ("n_objects", ctypes.c_int), ("edges", ctypes.c_void_p), ("counts", ctypes.c_void_p)]


class WsTileC(ctypes.Structure):
    _fields_ = [("labels", ctypes.c_void_p), ("edt", ctypes.c_void_p), ("W", ctypes.c_int), ("H", ctypes.c_int),
                ("n_objects", ctypes.c_int), ("out", ctypes.c_void_p), ("n_basins", ctypes.c_void_p)]


class Pipe:
    """A pipe_t handle.  Tensors passed in must be contiguous CUDA tensors
    on the pipe's device; calls are asynchronous on the given (or current)
    torch stream."""

    def __init__(self, device=0, params=None, **overrides):
        p = params if params is not None else default_params()
        for k, v in overrides.items():
            if k == "autotune_cache" and isinstance(v, str):
                v = v.encode()
                self._cache_path = v  # keeps the bytes alive while the pipe reads them
            setattr(p, k, v)
        self.params = p
        h = ctypes.c_void_p()
        _check(lib().pipe_create(ctypes.byref(p), device, ctypes.byref(h)), "pipe_create")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            lib().pipe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- plain form -------------------------------------------------------
    def seg_tile(self, rgb, hem8, labels, edt, n_objects, stream=None, pitch=None):
        H, W = rgb.shape[0], rgb.shape[1]
        pitch = pitch if pitch is not None else rgb.stride(0) * rgb.element_size()
        rc = lib().seg_tile(self.h, rgb.data_ptr(), W, H, pitch, hem8.data_ptr(), labels.data_ptr(),
                            edt.data_ptr() if edt is not None else None, n_objects.data_ptr(),
                            _stream_ptr(stream))
        _check(rc, "seg_tile")

    def features_tile(self, hem8, labels, n_objects, feats, stream=None):
        H, W = labels.shape
        rc = lib().features_tile(self.h, hem8.data_ptr(), labels.data_ptr(), W, H, int(n_objects),
                                 feats.data_ptr() if feats is not None else None, _stream_ptr(stream))
        _check(rc, "features_tile")

    def morph_open(self, src, dst, radius=9, stream=None):
        """Opening of a (H, W) uint8 device tensor by the disk of the given
        radius (Table I "Morph. Open": 19x19 disk, radius 9) into dst."""
        H, W = src.shape
        if tuple(dst.shape) != (H, W) or not src.is_contiguous() or not dst.is_contiguous():
            raise ValueError("src and dst must be contiguous (H, W) uint8 planes")
        rc = lib().morph_open_tile(self.h, src.data_ptr(), W, H, int(radius), dst.data_ptr(), _stream_ptr(stream))
        _check(rc, "morph_open_tile")

    def watershed(self, labels, edt, n_objects, out, n_basins, h=1, stream=None):
        """Watershed split of the labelled objects (Table I "Pre-Watershed" +
        "Watershed"): labels, edt and out are contiguous (H, W) int32 device
        tensors, n_basins a one-element int32 device tensor."""
        H, W = labels.shape
        for t in (labels, edt, out):
            if tuple(t.shape) != (H, W) or not t.is_contiguous():
                raise ValueError("labels, edt and out must be contiguous (H, W) int32 planes")
        rc = lib().watershed_tile(self.h, labels.data_ptr(), edt.data_ptr(), W, H, int(n_objects), int(h),
                                  out.data_ptr(), n_basins.data_ptr(), _stream_ptr(stream))
        _check(rc, "watershed_tile")

    def watershed_batch(self, tiles, h=1, stream=None):
        """tiles: list of dicts with labels, edt, out (contiguous (H, W) int32
        device tensors), n_objects (int) and n_basins (one-element int32
        device tensor)."""
        arr = (WsTileC * len(tiles))()
        for i, t in enumerate(tiles):
            H, W = t["labels"].shape
            for k in ("labels", "edt", "out"):
                if tuple(t[k].shape) != (H, W) or not t[k].is_contiguous():
                    raise ValueError("labels, edt and out must be contiguous (H, W) int32 planes")
            arr[i].labels, arr[i].edt, arr[i].out = t["labels"].data_ptr(), t["edt"].data_ptr(), t["out"].data_ptr()
            arr[i].W, arr[i].H, arr[i].n_objects = W, H, int(t["n_objects"])
            arr[i].n_basins = t["n_basins"].data_ptr()
        _check(lib().watershed_batch(self.h, arr, len(tiles), int(h), _stream_ptr(stream)), "watershed_batch")

    def rbc(self, rgb, out, t_lo=40, t_hi=100, stream=None, pitch=None):
        """Red blood cell mask (Table I "RBC detection") of an (H, W, 3) uint8
        device tensor into out, a contiguous (H, W) uint8 plane (0/1): the
        8-connected components of R - max(G, B) >= t_lo holding a pixel with
        R - max(G, B) >= t_hi."""
        H, W = rgb.shape[0], rgb.shape[1]
        if tuple(out.shape) != (H, W) or not out.is_contiguous():
            raise ValueError("out must be a contiguous (H, W) uint8 plane")
        pitch = pitch if pitch is not None else rgb.stride(0) * rgb.element_size()
        rc = lib().rbc_tile(self.h, rgb.data_ptr(), W, H, pitch, int(t_lo), int(t_hi), out.data_ptr(),
                            _stream_ptr(stream))
        _check(rc, "rbc_tile")

    def canny(self, img, edges, labels=None, n_objects=0, counts=None, low=40, high=120, radius=3, stream=None):
        """Canny edges of a (H, W) uint8 device tensor into edges (uint8 0/1),
        and, with labels (int32) and counts (int32 [n_objects]), the edge
        pixels within each object's disk dilation of the given radius."""
        H, W = img.shape
        if tuple(edges.shape) != (H, W) or not img.is_contiguous() or not edges.is_contiguous():
            raise ValueError("img and edges must be contiguous (H, W) uint8 planes")
        if labels is not None and (tuple(labels.shape) != (H, W) or not labels.is_contiguous()):
            raise ValueError("labels must be a contiguous (H, W) int32 plane")
        rc = lib().canny_tile(self.h, img.data_ptr(), labels.data_ptr() if labels is not None else None, W, H,
                              int(n_objects), int(low), int(high), int(radius), edges.data_ptr(),
                              counts.data_ptr() if counts is not None else None, _stream_ptr(stream))
        _check(rc, "canny_tile")

    def canny_batch(self, tiles, low=40, high=120, radius=3, stream=None):
        """tiles: list of dicts with img and edges (contiguous (H, W) uint8
        device tensors) and, optionally, labels ((H, W) int32), n_objects
        (int) and counts (int32 [n_objects])."""
        arr = (EdgeTileC * len(tiles))()
        for i, t in enumerate(tiles):
            H, W = t["img"].shape
            if tuple(t["edges"].shape) != (H, W) or not t["img"].is_contiguous() or not t["edges"].is_contiguous():
                raise ValueError("img and edges must be contiguous (H, W) uint8 planes")
            lab = t.get("labels")
            if lab is not None and (tuple(lab.shape) != (H, W) or not lab.is_contiguous()):
                raise ValueError("labels must be a contiguous (H, W) int32 plane")
            arr[i].img, arr[i].edges = t["img"].data_ptr(), t["edges"].data_ptr()
            arr[i].labels = lab.data_ptr() if lab is not None else None
            arr[i].W, arr[i].H, arr[i].n_objects = W, H, int(t.get("n_objects", 0))
            arr[i].counts = t["counts"].data_ptr() if t.get("counts") is not None else None
        _check(lib().canny_batch(self.h, arr, len(tiles), int(low), int(high), int(radius), _stream_ptr(stream)),
               "canny_batch")

    # ---- batched form ---------------------------------------------------
    def seg_features_batch(self, tiles, stream=None):
        """tiles: list of dicts with rgb, hem8, labels, edt, n_objects, feats (tensors)."""
        arr = (TileDevC * len(tiles))()
        for i, t in enumerate(tiles):
            rgb = t["rgb"]
            arr[i].rgb = rgb.data_ptr()
            arr[i].H, arr[i].W = rgb.shape[0], rgb.shape[1]
            arr[i].pitch = rgb.stride(0) * rgb.element_size()
            arr[i].hem8 = t["hem8"].data_ptr()
            arr[i].labels = t["labels"].data_ptr()
            arr[i].edt = t["edt"].data_ptr() if t.get("edt") is not None else None
            arr[i].n_objects = t["n_objects"].data_ptr()
            arr[i].feats = t["feats"].data_ptr()
            arr[i].feats_cap = t["feats"].shape[0]
        _check(lib().seg_features_batch(self.h, arr, len(tiles), _stream_ptr(stream)), "seg_features_batch")

    # ---- served form ----------------------------------------------------
    def submit(self, tiles, want_planes=False):
        """tiles: list of (H, W, 3) uint8 host arrays (numpy or pinned CPU
        tensors).  Returns a ticket, or None when admission is refused now."""
        arr = (TileDesc * len(tiles))()
        keep = []
        for i, t in enumerate(tiles):
            if hasattr(t, "data_ptr"):
                ptr, H, W, pitch = t.data_ptr(), t.shape[0], t.shape[1], t.stride(0)
            else:
                ptr, H, W, pitch = t.ctypes.data, t.shape[0], t.shape[1], t.strides[0]
            keep.append(t)
            arr[i].rgb_host, arr[i].W, arr[i].H, arr[i].pitch = ptr, W, H, pitch
            arr[i].want_planes = 1 if want_planes else 0
        tk = ctypes.c_uint64()
        rc = lib().batch_submit(self.h, arr, len(tiles), ctypes.byref(tk))
        if rc == PIPE_EBUSY:
            return None
        _check(rc, "batch_submit")
        self._keep = getattr(self, "_keep", {})
        self._keep[tk.value] = (keep, len(tiles), want_planes)
        return tk.value

    def poll(self, ticket):
        """None while the ticket runs; then a list of per-tile dicts (the
        results are copied out and the ticket released)."""
        import numpy as np
        keep, n, planes = self._keep[ticket]
        out = (TileResult * n)()
        nd = ctypes.c_int()
        rc = lib().batch_poll(self.h, ticket, ctypes.byref(nd), out)
        if rc == PIPE_EAGAIN:
            return None
        _check(rc, "batch_poll")
        res = []
        for i in range(n):
            r = out[i]
            H, W = keep[i].shape[0], keep[i].shape[1]
            rows = r.n_feats
            d = dict(status=r.status, n_objects=r.n_objects, t_arrive_ms=r.t_arrive_ms, t_done_ms=r.t_done_ms)
            d["feats"] = (np.ctypeslib.as_array(r.feats, (rows, NFEAT)).copy() if rows > 0 and r.feats
                          else np.zeros((0, NFEAT), np.float32))
            if planes:
                d["hem8"] = np.ctypeslib.as_array(r.hem8, (H, W)).copy()
                d["labels"] = np.ctypeslib.as_array(r.labels, (H, W)).copy()
                d["edt"] = np.ctypeslib.as_array(r.edt, (H, W)).copy()
            res.append(d)
        _check(lib().batch_release(self.h, ticket), "batch_release")
        del self._keep[ticket]
        return res

    def serve_memory(self):
        """Device bytes held by the served form's contexts (all, and those
        with a group in flight) and the number of contexts."""
        a, f, c = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int()
        _check(lib().pipe_serve_memory(self.h, ctypes.byref(a), ctypes.byref(f), ctypes.byref(c)),
               "pipe_serve_memory")
        return dict(allocated=a.value, in_flight=f.value, contexts=c.value)

    # ---- introspection --------------------------------------------------
    def status(self):
        return lib().pipe_status_read(self.h)

    def debug_plane(self, which, dst, stream=None):
        _check(lib().pipe_debug_plane(self.h, which, dst.data_ptr(), _stream_ptr(stream)), "pipe_debug_plane")

    def profile(self, enable):
        _check(lib().pipe_profile_enable(self.h, 1 if enable else 0), "pipe_profile_enable")

    def profile_read(self):
        cap = 64
        names = (ctypes.c_char_p * cap)()
        cnt = (ctypes.c_longlong * cap)()
        ms = (ctypes.c_double * cap)()
        n = lib().pipe_profile_read(self.h, names, cnt, ms, cap)
        return {names[i].decode(): (cnt[i], ms[i]) for i in range(min(n, cap))}

    def launch_count(self):
        return lib().pipe_launch_count(self.h)

    def recon_visits(self):
        return lib().pipe_recon_visits(self.h)

    def autotune_info(self):
        """Launch shapes of the latest batched call and the autotuner's timed
        passes so far: dict(recon_workers, edt_rows, feat_blocks, tune_runs)."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        r = ctypes.c_longlong()
        _check(lib().pipe_autotune_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(r)),
               "pipe_autotune_info")
        return dict(recon_workers=a.value, edt_rows=b.value, feat_blocks=c.value, tune_runs=r.value)
