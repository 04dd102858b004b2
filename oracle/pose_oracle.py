"""FP64 oracle of the pose gradients (test infrastructure; see package docstring).

The paper's method keeps the particle poses fixed (Sec. 4.1) and names joint pose
optimization as future work (Sec. 5).  The gradients it would need follow from the same
chain as App. A.2 Eqs. 16-21, one step earlier:

* mu_dot = W mu and Sigma_dot = W Sigma W^T (Sec. 3.3.2 Eq. 6), so for one particle
  dL/dW = sum_g [ grad_mu_dot mu^T + G W Sigma^T + G^T W Sigma ]
  with grad_mu_dot = [grad_mu_tilde; 0] and G = [[grad_Sigma_tilde, 0], [0, 0]] (Eq. 21),
  matrices differentiated as full matrices;
* an in-plane translation t of the model image moves every mu_tilde to mu_tilde + t, so
  dL/dt = sum_g grad_mu_tilde (at t = 0, the path's setting, Sec. 4.1).

grad_mu_tilde and grad_Sigma_tilde per (particle, Gaussian) are those of Eqs. 18-20, formed
here over each Gaussian's support exactly as ``gs_oracle.backward`` forms them.
"""
from __future__ import annotations

import numpy as np

from . import gs_oracle as O

F64 = np.float64
F32 = np.float32


def pose_backward(theta, Ws, D, dLdQ, E=0.5, cutoff=3.0, boxes=None):
    """(dL/dW[B, 3, 3], dL/dt[B, 2]) for upstream dL/dQ[B, D, D]."""
    theta = np.asarray(theta, dtype=F64).reshape(-1, 11)
    Ws = np.asarray(Ws, dtype=F64).reshape(-1, 3, 3)
    g = O.build_gaussians(theta)
    N = theta.shape[0]
    rx, ry = O.pixel_centres(D, E)
    B = Ws.shape[0]
    dW = np.zeros((B, 3, 3))
    dt = np.zeros((B, 2))
    for b in range(B):
        W = Ws[b]
        mu_dot, Sigma_dot = O.viewing_transform(g["mu"], g["Sigma"], W)
        mu_t, Sigma_t = O.projection(mu_dot, Sigma_dot)
        if boxes is None:
            x0, x1, y0, y1 = O.support_fp32(theta.astype(F32), W.astype(F32), D, E, cutoff)[:4]
        else:
            x0, x1, y0, y1 = boxes[b]
        for n in range(N):
            if x0[n] > x1[n] or y0[n] > y1[n]:
                continue
            sl = (slice(y0[n], y1[n] + 1), slice(x0[n], x1[n] + 1))
            r = np.stack([rx[sl], ry[sl]], axis=-1)
            Gt = O.splat(r, mu_t[n], Sigma_t[n])
            wgt = dLdQ[b][sl] * g["A"][n] * Gt
            P = np.linalg.inv(Sigma_t[n])
            d = r - mu_t[n]
            gmu_t = P @ np.einsum("ij,ija->a", wgt, d)
            gPinv = 0.5 * (np.sum(wgt) * Sigma_t[n] - np.einsum("ij,ija,ijb->ab", wgt, d, d))
            G = np.zeros((3, 3))
            G[0:2, 0:2] = -P.T @ gPinv @ P.T
            gmu_dot = np.array([gmu_t[0], gmu_t[1], 0.0])
            S = g["Sigma"][n]
            dW[b] += np.outer(gmu_dot, g["mu"][n]) + G @ W @ S.T + G.T @ W @ S
            dt[b] += gmu_t
    return dW, dt
