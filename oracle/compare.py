"""Error metrics between a CUDA result and the FP64 oracle (test infrastructure).

Track parameters: |g - o| / max(|o|, floor) per component, with floors
(1 cm, 1 cm, 1 cm, 1e-3 1/GeV, 1e-2 rad, 1e-2 rad) so that values near zero
are judged on an absolute scale; phi is compared as an angular difference.
Covariance: |g - o| / sqrt(o_ii o_jj), i.e. relative to the correlation
scale of the pair, so that near-zero off-diagonal entries are not judged
relative to themselves; where o_ii o_jj = 0 (the z row after a p2z step)
the entry must be exactly zero.  Bounds: 1e-4 on parameters, 1e-3 on
covariance elements.

A track on a cylinder has no variance along the surface normal, so its
Cartesian (x, y) block is singular along a direction set by the crossing
angle; an element such as C_xx = sin^2(a) C_tt is then as sensitive to a as
1/a.  For such tracks the covariances are compared in the surface frame
(t, r, z, k, phi, theta) of the oracle's crossing point, where the radial
row is compared against the tangential scale.
"""
from __future__ import annotations

import math

import numpy as np

PARAM_FLOORS = np.array([1.0, 1.0, 1.0, 1e-3, 1e-2, 1e-2])
TOL_PARAM = 1e-4
TOL_COV = 1e-3
_TRI = [(i, j) for i in range(6) for j in range(i + 1)]
_DIAG = [i * (i + 1) // 2 + i for i in range(6)]


def param_errors(g: np.ndarray, o: np.ndarray) -> np.ndarray:
    """g, o: [n, 6] -> relative errors [n, 6]."""
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    d = np.abs(g - o)
    d[:, 4] = np.abs((g[:, 4] - o[:, 4] + math.pi) % (2 * math.pi) - math.pi)
    return d / np.maximum(np.abs(o), PARAM_FLOORS)


def cov_errors(g: np.ndarray, o: np.ndarray) -> np.ndarray:
    """g, o: [n, 21] packed -> errors relative to sqrt(o_ii o_jj), [n, 21]."""
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    diag = o[:, _DIAG]
    scale = np.stack([np.sqrt(np.abs(diag[:, i] * diag[:, j])) for i, j in _TRI], axis=1)
    d = np.abs(g - o)
    with np.errstate(divide="ignore", invalid="ignore"):
        err = np.where(scale > 0, d / np.where(scale > 0, scale, 1.0), np.where(d == 0, 0.0, np.inf))
    return err


def unpack(c21: np.ndarray) -> np.ndarray:
    """[n, 21] -> [n, 6, 6]."""
    c21 = np.asarray(c21, dtype=np.float64)
    out = np.empty((c21.shape[0], 6, 6))
    k = 0
    for i in range(6):
        for j in range(i + 1):
            out[:, i, j] = out[:, j, i] = c21[:, k]
            k += 1
    return out


def pack(C: np.ndarray) -> np.ndarray:
    return np.stack([C[:, i, j] for i, j in _TRI], axis=1)


def surface_frame(cov: np.ndarray, angle: np.ndarray) -> np.ndarray:
    """Rotate packed covariances [n, 21] so that components 0, 1 become the
    tangential and radial position coordinates at azimuth `angle`."""
    C = unpack(cov)
    Q = np.tile(np.eye(6), (C.shape[0], 1, 1))
    s, c = np.sin(angle), np.cos(angle)
    Q[:, 0, 0], Q[:, 0, 1], Q[:, 1, 0], Q[:, 1, 1] = -s, c, c, s
    return pack(np.einsum("nij,njk,nlk->nil", Q, C, Q))


def cov_errors_frame(g: np.ndarray, o: np.ndarray, angle: np.ndarray) -> np.ndarray:
    """Covariance errors in the surface frame at `angle` (radial row judged on
    the tangential scale)."""
    gf, of = surface_frame(g, angle), surface_frame(o, angle)
    diag = of[:, _DIAG].copy()
    diag[:, 1] = diag[:, 0]  # the radial variance is structurally zero
    scale = np.stack([np.sqrt(np.abs(diag[:, i] * diag[:, j])) for i, j in _TRI], axis=1)
    d = np.abs(gf - of)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(scale > 0, d / np.where(scale > 0, scale, 1.0), np.where(d == 0, 0.0, np.inf))


def summary(err: np.ndarray) -> dict:
    if err.size == 0:
        return {"max": 0.0, "p99": 0.0, "mean": 0.0}
    flat = err.reshape(-1)
    return {"max": float(flat.max()), "p99": float(np.percentile(flat, 99)),
            "mean": float(flat.mean())}


def compare(g_state, g_cov, g_status, o_state, o_cov, o_status,
            tol_param: float = TOL_PARAM, tol_cov: float = TOL_COV,
            on_cylinder=None) -> dict:
    """All arrays per track ([n, 6], [n, 21], [n]).  Returns a report dict with
    'ok', error summaries per component and the status agreement.
    on_cylinder: bool [n], tracks whose covariances are compared in the
    surface frame of the oracle's point."""
    g_status = np.asarray(g_status).astype(np.int64)
    o_status = np.asarray(o_status).astype(np.int64)
    pe = param_errors(g_state, o_state)
    ce = cov_errors(g_cov, o_cov)
    if on_cylinder is not None and np.any(on_cylinder):
        m = np.asarray(on_cylinder, dtype=bool)
        os_ = np.asarray(o_state, dtype=np.float64)
        ang = np.arctan2(os_[m, 1], os_[m, 0])
        ce[m] = cov_errors_frame(np.asarray(g_cov)[m], np.asarray(o_cov)[m], ang)
    status_equal = bool(np.array_equal(g_status, o_status))
    rep = {
        "n": int(len(o_status)),
        "status_equal": status_equal,
        "status_mismatch": int(np.sum(g_status != o_status)),
        "flagged": int(np.sum(o_status != 0)),
        "param": summary(pe),
        "param_by_component": [summary(pe[:, c]) for c in range(6)],
        "cov": summary(ce),
        "tol_param": tol_param,
        "tol_cov": tol_cov,
    }
    rep["ok"] = bool(status_equal and rep["param"]["max"] <= tol_param
                     and rep["cov"]["max"] <= tol_cov)
    if not rep["ok"] and len(o_status):
        # the worst tracks and the status mismatches, to make a failure
        # readable (and recordable) on its own
        g_state = np.asarray(g_state)
        g_cov = np.asarray(g_cov)
        tp = int(np.argmax(pe.max(axis=1)))
        tc = int(np.argmax(ce.max(axis=1)))
        ec = int(np.argmax(ce[tc]))
        rep["worst_param"] = {"track": tp, "component": int(np.argmax(pe[tp])),
                              "err": pe[tp].tolist(), "gpu": g_state[tp].tolist(),
                              "oracle": np.asarray(o_state)[tp].tolist(),
                              "status_gpu": int(g_status[tp]), "status_oracle": int(o_status[tp])}
        rep["worst_cov"] = {"track": tc, "element": ec, "err": ce[tc].tolist(),
                            "gpu": g_cov[tc].tolist(), "oracle": np.asarray(o_cov)[tc].tolist(),
                            "status_gpu": int(g_status[tc]), "status_oracle": int(o_status[tc])}
        bad = np.nonzero(g_status != o_status)[0][:10]
        rep["status_mismatch_tracks"] = bad.tolist()
        rep["status_mismatch_values"] = [[int(g_status[t]), int(o_status[t])] for t in bad]
        rep["tracks_over_bound"] = int(np.sum((pe.max(axis=1) > tol_param)
                                              | (ce.max(axis=1) > tol_cov)))
    return rep
