"""CPU oracle for the rest of the training step on the device: the two
auxiliary terms of Eq. 17 that need no extra supervision (transmittance
concentration L_Tc and total variation L_tv on the density field) and the
Adam update of the voxel parameters with the optimizer re-initialisation of
Sec. IV-D.  Plain numpy in FP64.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and the CPU-baseline leg of
``bench.py``; never by the product package.

Readings (the paper names the terms, not their formulas):
  - L_Tc "encourages final ray transmittance to be near 0 or 1" (Eq. 17):
    L_Tc = lambda / |P| * sum_p T_p (1 - T_p), zero at both ends, largest at
    T = 1/2; dL/dT_p = lambda (1 - 2 T_p) / |P|.
  - L_tv is "total variation on the sparse density field" (Eq. 17); with 8
    corner densities per voxel the field inside a voxel is their trilinear
    interpolant, and its variation is measured along the 12 cube edges:
    L_tv = lambda / N * sum_v sum_{edges (i, j)} (d_i - d_j)^2, corner index
    c = x + 2 y + 4 z, edges join corners that differ in one bit;
    dL/dd_i = 2 lambda / N * sum_{j adjacent to i} (d_i - d_j).
  - Adam (the optimizer refreshed after topology changes, Sec. IV-D):
    m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
    p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), one global
    step count t; children start from m = v = 0 (the subdivision fills them).
"""
from __future__ import annotations

import numpy as np

# the 12 edges of the corner cube: (c, c | bit) for every bit not set in c
EDGES = [(c, c | b) for b in (1, 2, 4) for c in range(8) if not c & b]


def transmittance_concentration(T, weight):
    """L_Tc and dL/dT (Eq. 17, reading above)."""
    T = np.asarray(T, np.float64)
    P = T.size
    if P == 0:
        return 0.0, np.zeros(0)
    loss = weight * float(np.sum(T * (1.0 - T))) / P
    return loss, weight * (1.0 - 2.0 * T) / P


def density_tv(density, weight):
    """L_tv over the 12 edges of each voxel's corner cube and its gradient."""
    d = np.asarray(density, np.float64).reshape(-1, 8)
    n = d.shape[0]
    if n == 0:
        return 0.0, np.zeros((0, 8))
    loss = 0.0
    grad = np.zeros_like(d)
    for i, j in EDGES:
        diff = d[:, i] - d[:, j]
        loss += float(np.sum(diff * diff))
        grad[:, i] += 2.0 * diff
        grad[:, j] -= 2.0 * diff
    return weight * loss / n, weight * grad / n


def adam(param, grad, m, v, lr, beta1, beta2, eps, step):
    """One Adam update; returns (param, m, v) as new FP64 arrays."""
    p = np.asarray(param, np.float64)
    g = np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def adam_voxels(density, sh, d_density, d_sh, m_d, v_d, m_s, v_s, lr_density, lr_sh, beta1, beta2, eps, step,
                tv_weight=0.0):
    """The voxel update: density gradient plus the L_tv gradient, then Adam on
    the corner densities and (when d_sh is given) on the SH coefficients."""
    tv, g_tv = density_tv(density, tv_weight)
    g = np.asarray(d_density, np.float64).reshape(-1, 8) + g_tv
    dens, m_d, v_d = adam(np.asarray(density, np.float64).reshape(-1, 8), g, m_d, v_d, lr_density, beta1, beta2,
                          eps, step)
    out = {"density": dens, "m_density": m_d, "v_density": v_d, "tv_loss": tv}
    if d_sh is not None:
        out["sh"], out["m_sh"], out["v_sh"] = adam(sh, d_sh, m_s, v_s, lr_sh, beta1, beta2, eps, step)
    return out
