"""Two-centre Slater-Koster blocks for an s/p/d minimal basis -- oracle, test-only.

The paper's copper model (Sec. II.A) builds each off-diagonal 9x9 block of H from ten bond
integrals and the direction cosines of the bond, following Slater & Koster, Phys. Rev. 94,
1498 (1954), Table I.  Every bond integral here carries the same radial factor
V_i * exp(-decay * (r / r0 - 1)).

Orbital order: s, px, py, pz, dxy, dyz, dzx, dx2-y2, d3z2-r2.  ``block(d)`` is the block
H_ab for d = R_b - R_a (row orbital on atom a, column orbital on atom b).  Entries with the
row orbital later in the order than the column orbital follow from the parity rule
E_{beta,alpha}(l, m, n) = (-1)^(L_alpha + L_beta) E_{alpha,beta}(l, m, n).

All arithmetic is written so that complex ``d`` works, which gives dH/dd to machine precision
by the complex-step method (Squire & Trapp, SIAM Rev. 40, 110 (1998)).
"""
from __future__ import annotations

import numpy as np

_ANG = np.array([0, 1, 1, 1, 2, 2, 2, 2, 2])
_S3 = np.sqrt(3.0)


def block(d: np.ndarray, V, r0: float, decay: float) -> np.ndarray:
    """SK blocks for bond vectors d of shape (B, 3) (real or complex) -> (B, 9, 9)."""
    d = np.asarray(d)
    dx, dy, dz = d[:, 0], d[:, 1], d[:, 2]
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    l, m, n = dx / r, dy / r, dz / r
    rad = np.exp(-decay * (r / r0 - 1.0))
    sss, sps, sds, pps, ppp, pds, pdp, dds, ddp, ddd = [v * rad for v in V]
    l2, m2, n2 = l * l, m * m, n * n
    E = np.zeros((d.shape[0], 9, 9), dtype=np.result_type(d.dtype, np.float64))
    # s-s, s-p, s-d
    E[:, 0, 0] = sss
    E[:, 0, 1] = l * sps
    E[:, 0, 2] = m * sps
    E[:, 0, 3] = n * sps
    E[:, 0, 4] = _S3 * l * m * sds
    E[:, 0, 5] = _S3 * m * n * sds
    E[:, 0, 6] = _S3 * n * l * sds
    E[:, 0, 7] = 0.5 * _S3 * (l2 - m2) * sds
    E[:, 0, 8] = (n2 - 0.5 * (l2 + m2)) * sds
    # p-p
    E[:, 1, 1] = l2 * pps + (1.0 - l2) * ppp
    E[:, 1, 2] = l * m * (pps - ppp)
    E[:, 1, 3] = l * n * (pps - ppp)
    E[:, 2, 2] = m2 * pps + (1.0 - m2) * ppp
    E[:, 2, 3] = m * n * (pps - ppp)
    E[:, 3, 3] = n2 * pps + (1.0 - n2) * ppp
    # p-d
    E[:, 1, 4] = _S3 * l2 * m * pds + m * (1.0 - 2.0 * l2) * pdp
    E[:, 1, 5] = _S3 * l * m * n * pds - 2.0 * l * m * n * pdp
    E[:, 1, 6] = _S3 * l2 * n * pds + n * (1.0 - 2.0 * l2) * pdp
    E[:, 1, 7] = 0.5 * _S3 * l * (l2 - m2) * pds + l * (1.0 - l2 + m2) * pdp
    E[:, 1, 8] = l * (n2 - 0.5 * (l2 + m2)) * pds - _S3 * l * n2 * pdp
    E[:, 2, 4] = _S3 * m2 * l * pds + l * (1.0 - 2.0 * m2) * pdp
    E[:, 2, 5] = _S3 * m2 * n * pds + n * (1.0 - 2.0 * m2) * pdp
    E[:, 2, 6] = _S3 * l * m * n * pds - 2.0 * l * m * n * pdp
    E[:, 2, 7] = 0.5 * _S3 * m * (l2 - m2) * pds - m * (1.0 + l2 - m2) * pdp
    E[:, 2, 8] = m * (n2 - 0.5 * (l2 + m2)) * pds - _S3 * m * n2 * pdp
    E[:, 3, 4] = _S3 * l * m * n * pds - 2.0 * l * m * n * pdp
    E[:, 3, 5] = _S3 * n2 * m * pds + m * (1.0 - 2.0 * n2) * pdp
    E[:, 3, 6] = _S3 * n2 * l * pds + l * (1.0 - 2.0 * n2) * pdp
    E[:, 3, 7] = 0.5 * _S3 * n * (l2 - m2) * pds - n * (l2 - m2) * pdp
    E[:, 3, 8] = n * (n2 - 0.5 * (l2 + m2)) * pds + _S3 * n * (l2 + m2) * pdp
    # d-d
    E[:, 4, 4] = 3.0 * l2 * m2 * dds + (l2 + m2 - 4.0 * l2 * m2) * ddp + (n2 + l2 * m2) * ddd
    E[:, 4, 5] = 3.0 * l * m2 * n * dds + l * n * (1.0 - 4.0 * m2) * ddp + l * n * (m2 - 1.0) * ddd
    E[:, 4, 6] = 3.0 * l2 * m * n * dds + m * n * (1.0 - 4.0 * l2) * ddp + m * n * (l2 - 1.0) * ddd
    E[:, 4, 7] = (1.5 * l * m * (l2 - m2) * dds + 2.0 * l * m * (m2 - l2) * ddp
                  + 0.5 * l * m * (l2 - m2) * ddd)
    E[:, 4, 8] = (_S3 * l * m * (n2 - 0.5 * (l2 + m2)) * dds - 2.0 * _S3 * l * m * n2 * ddp
                  + 0.5 * _S3 * l * m * (1.0 + n2) * ddd)
    E[:, 5, 5] = 3.0 * m2 * n2 * dds + (m2 + n2 - 4.0 * m2 * n2) * ddp + (l2 + m2 * n2) * ddd
    E[:, 5, 6] = 3.0 * m * n2 * l * dds + m * l * (1.0 - 4.0 * n2) * ddp + m * l * (n2 - 1.0) * ddd
    E[:, 5, 7] = (1.5 * m * n * (l2 - m2) * dds - m * n * (1.0 + 2.0 * (l2 - m2)) * ddp
                  + m * n * (1.0 + 0.5 * (l2 - m2)) * ddd)
    E[:, 5, 8] = (_S3 * m * n * (n2 - 0.5 * (l2 + m2)) * dds + _S3 * m * n * (l2 + m2 - n2) * ddp
                  - 0.5 * _S3 * m * n * (l2 + m2) * ddd)
    E[:, 6, 6] = 3.0 * n2 * l2 * dds + (n2 + l2 - 4.0 * n2 * l2) * ddp + (m2 + n2 * l2) * ddd
    E[:, 6, 7] = (1.5 * n * l * (l2 - m2) * dds + n * l * (1.0 - 2.0 * (l2 - m2)) * ddp
                  - n * l * (1.0 - 0.5 * (l2 - m2)) * ddd)
    E[:, 6, 8] = (_S3 * l * n * (n2 - 0.5 * (l2 + m2)) * dds + _S3 * l * n * (l2 + m2 - n2) * ddp
                  - 0.5 * _S3 * l * n * (l2 + m2) * ddd)
    E[:, 7, 7] = (0.75 * (l2 - m2) ** 2 * dds + (l2 + m2 - (l2 - m2) ** 2) * ddp
                  + (n2 + 0.25 * (l2 - m2) ** 2) * ddd)
    E[:, 7, 8] = (0.5 * _S3 * (l2 - m2) * (n2 - 0.5 * (l2 + m2)) * dds
                  + _S3 * n2 * (m2 - l2) * ddp + 0.25 * _S3 * (1.0 + n2) * (l2 - m2) * ddd)
    E[:, 8, 8] = ((n2 - 0.5 * (l2 + m2)) ** 2 * dds + 3.0 * n2 * (l2 + m2) * ddp
                  + 0.75 * (l2 + m2) ** 2 * ddd)
    # lower triangle by parity
    for a in range(9):
        for b in range(a):
            E[:, a, b] = (-1.0) ** (_ANG[a] + _ANG[b]) * E[:, b, a]
    return E


def block_grad(d: np.ndarray, V, r0: float, decay: float, h: float = 1e-30) -> np.ndarray:
    """dH_ab/dd_c for bond vectors d (B, 3) -> (B, 3, 9, 9), by the complex step."""
    d = np.asarray(d, dtype=np.float64)
    out = np.zeros((d.shape[0], 3, 9, 9))
    for c in range(3):
        dc = d.astype(np.complex128)
        dc[:, c] += 1j * h
        out[:, c] = block(dc, V, r0, decay).imag / h
    return out


def onsite_block(es: float, ep: float, ed: float) -> np.ndarray:
    return np.diag([es, ep, ep, ep, ed, ed, ed, ed, ed]).astype(np.float64)
