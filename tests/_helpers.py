"""Shared helpers of the test-suite (comparison metrics, cached oracle tables)."""
import hashlib
import os

import numpy as np

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CACHE = os.path.join(ROOT, "tests", ".cache")

# tolerances (the per-ray field is compared in relative L2 over the ray,
# composited pixels in max absolute error per channel)
FIELD_REL_L2 = 1e-5
PIXEL_ABS = 2e-4
TANGENCY_BAND = 1e-6  # in units of h


def oracle_lut(kernel, K, D, n_lambda):
    """The oracle's table, cached on disk (it is the oracle's own output)."""
    os.makedirs(CACHE, exist_ok=True)
    key = "lut_%s_K%d_D%d_N%d" % (kernel, K, D, n_lambda)
    path = os.path.join(CACHE, key + ".npz")
    src = open(os.path.join(ROOT, "oracle", "oracle.c"), "rb").read()
    tag = hashlib.sha1(src).hexdigest()[:12]
    if os.path.exists(path):
        z = np.load(path)
        if str(z["tag"]) == tag:
            return dict(kernel=oracle.KERNELS[kernel], K=K, D=D, n_lambda=n_lambda, q=float(z["q"]),
                        theta=z["theta"], pieces=z["pieces"], err=z["err"], normB=z["normB"], integ=z["integ"],
                        lam=z["lam"])
    L = oracle.lut_build(kernel, K, D, n_lambda)
    tmp = path + ".tmp%d.npz" % os.getpid()
    np.savez(tmp, tag=tag, q=L["q"], theta=L["theta"], pieces=L["pieces"], err=L["err"], normB=L["normB"],
             integ=L["integ"], lam=L["lam"])
    os.replace(tmp, path)
    return L


def field_rel_l2(rows_a, rows_b, D):
    """||F_a - F_b||_2 / ||F_b||_2 over the ray; rows are (t_a, t_b, A_0..A_D) of positive-length pieces,
    integrated exactly (Gauss-Legendre, 8 nodes) over the union of both sets of breakpoints."""
    ra = rows_a[rows_a[:, 1] > rows_a[:, 0]]
    rb = rows_b[rows_b[:, 1] > rows_b[:, 0]]
    if len(rb) == 0 and len(ra) == 0:
        return 0.0
    pts = np.unique(np.concatenate([ra[:, 0], ra[:, 1], rb[:, 0], rb[:, 1]]))
    x, w = np.polynomial.legendre.leggauss(8)
    a, b = pts[:-1], pts[1:]
    mid, half = 0.5 * (a + b), 0.5 * (b - a)
    t = (mid[:, None] + half[:, None] * x[None, :]).ravel()
    ww = (half[:, None] * w[None, :]).ravel()

    def ev(rows):
        out = np.zeros_like(t)
        if len(rows) == 0:
            return out
        idx = np.searchsorted(rows[:, 0], t, side="right") - 1
        ok = (idx >= 0) & (t <= rows[np.clip(idx, 0, None), 1])
        r = rows[np.clip(idx, 0, None)]
        y = t - r[:, 0]
        v = np.zeros_like(t)
        for d in range(D, -1, -1):
            v = v * y + r[:, 2 + d]
        out[ok] = v[ok]
        return out

    fa, fb = ev(ra), ev(rb)
    den = np.sqrt(np.sum(ww * fb * fb))
    num = np.sqrt(np.sum(ww * (fa - fb) ** 2))
    return num / den if den > 0 else num


def tangency_band(P, o, v, q, ids=None):
    """Indices of particles within TANGENCY_BAND * h of the kernel-support tangency for the ray (o, v)."""
    pos = P["pos"].astype(np.float64)
    h = P["h"].astype(np.float64)
    if ids is not None:
        pos, h = pos[ids], h[ids]
    x = pos - o
    tc = x @ v
    d = np.linalg.norm(x - tc[:, None] * v[None, :], axis=1)
    band = np.abs(d - q * h) <= TANGENCY_BAND * h
    idx = np.nonzero(band)[0]
    return set((ids[idx] if ids is not None else idx).tolist())
