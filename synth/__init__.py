"""Seeded synthetic RGB tiles: the shared input of the CUDA path and the oracle.

The generator (``synth.c``) paints background, stroma discs, an optional
serpentine ramp corridor and nuclei ellipses, then adds noise, blurs and
rounds.  It holds none of the segmentation or feature arithmetic.  The
workloads mirror the paper's 4Kx4K tiles (Sec. V-A) and its nuclei density
(Sec. II); the paper's own images are not available.

Workload presets (sizes, counts, seeds):

* ``cfg0()``  512x512, ~60 nuclei, 10% overlapping; seed 0.
* ``cfg1()``  4096x4096, ~3000 nuclei, 20% in touching clusters of 2-6, plus
  150 stroma discs of radius 40-120; seed 1000.
* ``cfg2(i)`` tile i of a 64-tile batch: side in {1024,2048,3072,4096},
  density uniform in [0,5000] nuclei per 4096^2 area; tile 0 empty, tile 1
  at 5000; seed 2000+i.
* ``cfg3(i)`` tile i of the 64-tile pool served by the request stream: side
  a multiple of 256 in [2048,4096], density as cfg2; seed 3000+i.
* ``cfg4(i)`` tile i of the 32-tile worst-case pool: 4096^2, 8000 nuclei,
  half of them in chains of 10-30, plus a ~3900 px serpentine ramp band;
  seed 4000+i.
"""
import ctypes
import os
import subprocess

import numpy as np

_here = os.path.dirname(os.path.abspath(__file__))
_lib = None


class SynthCfg(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int), ("H", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("n_nuclei", ctypes.c_int), ("frac_overlap", ctypes.c_double),
                ("frac_cluster", ctypes.c_double), ("frac_chain", ctypes.c_double),
                ("n_stroma", ctypes.c_int), ("stroma_rmin", ctypes.c_double),
                ("stroma_rmax", ctypes.c_double), ("corridor", ctypes.c_int), ("n_rbc", ctypes.c_int)]


def build(force=False):
    """Compile libsynth.so next to this file (gcc, OpenMP)."""
    so = os.path.join(_here, "libsynth.so")
    src = os.path.join(_here, "synth.c")
    hdr = os.path.join(_here, "synth.h")
    if force or not os.path.exists(so) or os.path.getmtime(so) < max(os.path.getmtime(src), os.path.getmtime(hdr)):
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-o", so, src, "-lm"])
    return so


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.synth_tile.argtypes = [ctypes.POINTER(SynthCfg), ctypes.c_void_p, ctypes.c_size_t]
        _lib.synth_tile.restype = ctypes.c_int
    return _lib


def tile(W, H, seed, n_nuclei=0, frac_overlap=0.0, frac_cluster=0.0, frac_chain=0.0,
         n_stroma=0, stroma_rmin=40.0, stroma_rmax=120.0, corridor=False, n_rbc=0):
    """Return an (H, W, 3) uint8 RGB tile."""
    cfg = SynthCfg(W, H, seed, n_nuclei, frac_overlap, frac_cluster, frac_chain, n_stroma,
                   stroma_rmin, stroma_rmax, 1 if corridor else 0, n_rbc)
    out = np.empty((H, W, 3), np.uint8)
    rc = _load().synth_tile(ctypes.byref(cfg), out.ctypes.data, W * 3)
    if rc != 0:
        raise RuntimeError("synth_tile failed with code %d" % rc)
    return out


def _density_tile(side, density, seed):
    n = int(round(density * side * side / 4096.0 ** 2))
    return tile(side, side, seed, n_nuclei=n, frac_overlap=0.1, frac_cluster=0.2,
                n_stroma=int(round(0.05 * n)))


def cfg0():
    return tile(512, 512, 0, n_nuclei=60, frac_overlap=0.1)


def cfg1():
    return tile(4096, 4096, 1000, n_nuclei=3000, frac_overlap=0.0, frac_cluster=0.2,
                n_stroma=150)


def _sm64(z):
    """SplitMix64 output function (Steele, Lea, Flood 2014)."""
    m = (1 << 64) - 1
    z = (z + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def _draw(seed, i):
    """Two uniform numbers in [0,1) for tile i, independent of the pixel draws."""
    a = _sm64(_sm64(seed * 1000003 + 2 * i))
    b = _sm64(_sm64(seed * 1000003 + 2 * i + 1))
    return (a >> 11) / float(1 << 53), (b >> 11) / float(1 << 53)


def cfg2_shape(i):
    """(side, density) of batch tile i."""
    u, v = _draw(2999, i)
    side = (1024, 2048, 3072, 4096)[min(3, int(u * 4))]
    density = 5000.0 * v
    if i == 0:
        density = 0.0
    if i == 1:
        density = 5000.0
    return side, density


def cfg2(i):
    side, density = cfg2_shape(i)
    return _density_tile(side, density, 2000 + i)


def cfg3_shape(i):
    u, v = _draw(3998, i)
    side = 256 * (8 + min(8, int(u * 9)))
    return side, 5000.0 * v


def cfg3(i):
    side, density = cfg3_shape(i)
    return _density_tile(side, density, 3000 + i)


def cfg4(i):
    return tile(4096, 4096, 4000 + i, n_nuclei=8000, frac_chain=0.5, n_stroma=0, corridor=True)
