"""Brute-force restatements of each step's definition, used to pin the oracle.

Written independently of oracle/oracle.c: different algorithms (iterated
dilation instead of Vincent's queue, union-find instead of BFS, all-pairs
distances instead of Meijster's envelope, numpy formulas for features) so
that a slip in one is not repeated in the other.  Small inputs only.
"""
import math

import numpy as np

OFFSETS = ((1, 0), (0, 1), (1, 1), (1, -1))  # (dx, dy)


# ---- colour deconvolution -------------------------------------------------

def deconv_constants():
    H = np.array([0.650, 0.704, 0.286])
    E = np.array([0.072, 0.990, 0.105])
    H = H / np.linalg.norm(H)
    E = E / np.linalg.norm(E)
    R = np.cross(H, E)
    R = R / np.linalg.norm(R)
    w = np.linalg.inv(np.stack([H, E, R]))[:, 0]
    lut = [math.floor(-math.log((v + 1) / 256.0) * 256.0 + 0.5) for v in range(256)]
    wq = [int(round(100.0 * x * 2048.0)) for x in w]
    return np.array(lut, np.int64), np.array(wq, np.int64), w


def deconv(rgb):
    lut, wq, _ = deconv_constants()
    acc = wq[0] * lut[rgb[..., 0]] + wq[1] * lut[rgb[..., 1]] + wq[2] * lut[rgb[..., 2]]
    v = np.where(acc < 0, 0, (acc + (1 << 18)) >> 19)
    return np.minimum(v, 255).astype(np.uint8)


# ---- reconstruction --------------------------------------------------------

def dilate8(a):
    """3x3 max; outside pixels ignored (padding with 0 is the same for a>=0)."""
    p = np.pad(a, 1, constant_values=0)
    H, W = a.shape
    out = np.zeros_like(a)
    for dy in (0, 1, 2):
        for dx in (0, 1, 2):
            out = np.maximum(out, p[dy:dy + H, dx:dx + W])
    return out


def recon_iterated(marker, mask):
    """R_{k+1} = min(dilate8(R_k), mask) until stable; returns (R, iterations)."""
    R = marker.astype(np.int32)
    m = mask.astype(np.int32)
    it = 0
    while True:
        nx = np.minimum(dilate8(R), m)
        if np.array_equal(nx, R):
            return R.astype(np.uint8), it
        R = nx
        it += 1


def hdome_fg(hem8, h, thr):
    hem = hem8.astype(np.int32)
    marker = np.maximum(hem - h, 0)
    R, _ = recon_iterated(marker, hem)
    return R, (hem - R.astype(np.int32) >= thr).astype(np.uint8)


# ---- union-find helpers ----------------------------------------------------

class UF:
    def __init__(self, n):
        self.p = list(range(n))

    def find(self, a):
        while self.p[a] != a:
            self.p[a] = self.p[self.p[a]]
            a = self.p[a]
        return a

    def union(self, a, b):
        a, b = self.find(a), self.find(b)
        if a != b:
            if a < b:
                a, b = b, a
            self.p[a] = b


def components(mask, conn):
    """Union-find components of mask!=0; returns a root index per pixel (-1 off)."""
    H, W = mask.shape
    uf = UF(H * W)
    nb = [(0, -1), (-1, 0)] if conn == 4 else [(0, -1), (-1, -1), (-1, 0), (-1, 1)]
    for y in range(H):
        for x in range(W):
            if not mask[y, x]:
                continue
            for dy, dx in nb:
                yy, xx = y + dy, x + dx
                if 0 <= yy < H and 0 <= xx < W and mask[yy, xx]:
                    uf.union(y * W + x, yy * W + xx)
    root = np.full((H, W), -1, np.int64)
    for y in range(H):
        for x in range(W):
            if mask[y, x]:
                root[y, x] = uf.find(y * W + x)
    return root


def fill_holes(fg):
    H, W = fg.shape
    bg = fg == 0
    root = components(bg, 4)
    border = set()
    for y in range(H):
        for x in range(W):
            if bg[y, x] and (y in (0, H - 1) or x in (0, W - 1)):
                border.add(root[y, x])
    out = np.ones((H, W), np.uint8)
    for y in range(H):
        for x in range(W):
            if bg[y, x] and root[y, x] in border:
                out[y, x] = 0
    return out


def label(filled, amin, amax):
    H, W = filled.shape
    root = components(filled != 0, 8)
    area = {}
    for r in root[root >= 0].ravel():
        area[r] = area.get(r, 0) + 1
    # union-find roots are the smallest raster index of each component
    keep = sorted(r for r, a in area.items() if amin <= a <= amax)
    lab = {r: i + 1 for i, r in enumerate(keep)}
    out = np.zeros((H, W), np.int32)
    for y in range(H):
        for x in range(W):
            r = root[y, x]
            if r >= 0 and r in lab:
                out[y, x] = lab[r]
    return out, len(keep)


# ---- EDT -------------------------------------------------------------------

def edt_allpairs(labels):
    H, W = labels.shape
    ys, xs = np.nonzero(labels == 0)
    if len(ys) == 0:
        return np.full((H, W), 2 ** 31 - 1, np.int64)
    gy, gx = np.mgrid[0:H, 0:W]
    best = np.full((H, W), np.iinfo(np.int64).max, np.int64)
    for y, x in zip(ys, xs):
        best = np.minimum(best, (gy - y) ** 2 + (gx - x) ** 2)
    return best


# ---- features --------------------------------------------------------------

def sobel_m2(hem8):
    a = np.pad(hem8.astype(np.int64), 1, mode="edge")
    H, W = hem8.shape
    s = lambda dy, dx: a[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
    gx = (s(-1, 1) + 2 * s(0, 1) + s(1, 1)) - (s(-1, -1) + 2 * s(0, -1) + s(1, -1))
    gy = (s(1, -1) + 2 * s(1, 0) + s(1, 1)) - (s(-1, -1) + 2 * s(-1, 0) + s(-1, 1))
    return gx * gx + gy * gy


def glcm_stats(C):
    """contrast, energy, homogeneity, entropy, correlation of count matrix C."""
    T = C.sum()
    P = C / T
    i, j = np.mgrid[0:8, 0:8]
    con = float(((i - j) ** 2 * P).sum())
    ene = float((P ** 2).sum())
    hom = float((P / (1 + (i - j) ** 2)).sum())
    nz = P > 0
    ent = float(-(P[nz] * np.log(P[nz])).sum())
    # exact zero-variance detection with rational moments
    from fractions import Fraction
    Ci = [[int(C[a, b]) for b in range(8)] for a in range(8)]
    mu_i = Fraction(sum(a * Ci[a][b] for a in range(8) for b in range(8)), int(T))
    mu_j = Fraction(sum(b * Ci[a][b] for a in range(8) for b in range(8)), int(T))
    vi = sum((a - mu_i) ** 2 * Ci[a][b] for a in range(8) for b in range(8))
    vj = sum((b - mu_j) ** 2 * Ci[a][b] for a in range(8) for b in range(8))
    cv = sum((a - mu_i) * (b - mu_j) * Ci[a][b] for a in range(8) for b in range(8))
    cor = 0.0 if vi == 0 or vj == 0 else float(cv) / math.sqrt(float(vi) * float(vj))
    return np.array([con, ene, hom, ent, cor])


def features(hem8, labels, K):
    H, W = labels.shape
    m2 = sobel_m2(hem8)
    out = np.zeros((K, 15))
    for l in range(1, K + 1):
        om = labels == l
        N = int(om.sum())
        if N == 0:
            continue
        v = hem8[om].astype(np.float64)
        g = np.sqrt(m2[om].astype(np.float64))
        pad = np.pad(om, 1, constant_values=False)
        per = 0
        for dy, dx in ((-1, 0), (1, 0), (0, -1), (0, 1)):
            nb = pad[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
            per += int((om & ~nb).sum())
        stats = []
        for dx, dy in OFFSETS:
            C = np.zeros((8, 8), np.int64)
            for y in range(H):
                for x in range(W):
                    yy, xx = y + dy, x + dx
                    if om[y, x] and 0 <= yy < H and 0 <= xx < W and om[yy, xx]:
                        C[hem8[y, x] >> 5, hem8[yy, xx] >> 5] += 1
            if C.sum() > 0:
                stats.append(glcm_stats(C))
        tex = np.mean(stats, axis=0) if stats else np.zeros(5)
        out[l - 1] = [N, per, v.mean(), v.std(), v.min(), v.max(), g.mean(), g.std(), g.min(),
                      g.max(), *tex]
    return out
