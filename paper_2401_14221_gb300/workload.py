"""Seeded synthetic workloads for the p2z / p2r Kalman step.

The paper's mini-apps run on synthetic inputs: a fixed set of track parameters
smeared at random and reused for every track, grouped in events of equal track
count (section 2).  This module makes inputs of that shape with the sizes and
distributions of the benchmark workloads.  It holds none of the method's
arithmetic (no closed-form helix, no Jacobian, no Kalman algebra): the true
trajectory that places each hit on its surface is a *simulation* of the
particle, a fourth-order Runge-Kutta integration of the Lorentz force
d(t)/ds = q c k (t x B) written from the force law, with the unit constant
taken from the speed of light.  Both the oracle and the CUDA path read the
arrays made here; neither imports the other.

Canonical layout produced here: structure-of-arrays float32, one row per
component: state [6, n] = (x, y, z, 1/pT, phi, theta), cov [21, n] packed
lower-triangular (00, 10, 11, 20, 21, 22, ...), hit [3, n], hitcov [6, n]
packed 3x3, charge [n] int8.  ``to_aosoa``/``from_aosoa`` re-block these for
the array-of-structure-of-arrays layout (blocks of W tracks, section 2).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# Momentum (GeV/c) of a unit charge on a 1 cm radius orbit in 1 T: e*B*r
# expressed in GeV/c is B[T] * r[m] * c[m/s] * 1e-9.
SPEED_OF_LIGHT = 299_792_458.0
GEV_PER_T_CM = SPEED_OF_LIGHT * 1e-9 * 1e-2

# Per-component scale of the generated covariance (cm, cm, cm, 1/GeV, rad, rad);
# the 1/pT entry is relative (0.01 * k).
COV_SIGMA = (0.01, 0.01, 0.05, 0.01, 1e-3, 1e-3)

P2Z = 0
P2R = 1


def tri_index(i: int, j: int) -> int:
    if i < j:
        i, j = j, i
    return i * (i + 1) // 2 + j


@dataclasses.dataclass
class Workload:
    kind: int                      # P2Z or P2R
    n: int
    bz: float
    surf: object                   # z of the plane / r of the cylinder: float, or float32 [n]
    state: np.ndarray              # float32 [6, n] start state (smeared truth)
    cov: np.ndarray                # float32 [21, n]
    charge: np.ndarray             # int8 [n]
    hit: np.ndarray                # float32 [3, n]
    hitcov: np.ndarray             # float32 [6, n]
    truth_start: np.ndarray        # float64 [6, n]
    truth_surface: np.ndarray      # float64 [6, n] (nan where unreachable)
    reached: np.ndarray            # bool [n]: the true track reaches the surface
    events: int = 1
    description: str = ""


# --------------------------------------------------------------- simulation

def _rk4_deriv(tx, ty, kappa):
    # d(x, y)/ds = (tx, ty); d(tx, ty)/ds = kappa * (t x z_hat) = kappa * (ty, -tx)
    return tx, ty, kappa * ty, -kappa * tx


def rk4_transverse(x, y, tx, ty, kappa, h, steps: int):
    """Integrate the transverse motion with ``steps`` RK4 steps of size h
    (arrays, broadcast).  Returns (x, y, tx, ty)."""
    for _ in range(steps):
        k1 = _rk4_deriv(tx, ty, kappa)
        k2 = _rk4_deriv(tx + 0.5 * h * k1[2], ty + 0.5 * h * k1[3], kappa)
        k3 = _rk4_deriv(tx + 0.5 * h * k2[2], ty + 0.5 * h * k2[3], kappa)
        k4 = _rk4_deriv(tx + h * k3[2], ty + h * k3[3], kappa)
        x = x + h / 6.0 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        y = y + h / 6.0 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
        tx_n = tx + h / 6.0 * (k1[2] + 2 * k2[2] + 2 * k3[2] + k4[2])
        ty_n = ty + h / 6.0 * (k1[3] + 2 * k2[3] + 2 * k3[3] + k4[3])
        tx, ty = tx_n, ty_n
    return x, y, tx, ty


def curvature_rate(q, k, bz):
    """kappa in d(t)/ds = kappa (t x z_hat), from F = q v x B."""
    return np.asarray(q, dtype=np.float64) * GEV_PER_T_CM * bz * np.asarray(k, dtype=np.float64)


def simulate_to_z(truth: np.ndarray, q, bz: float, zt, steps: int = 64):
    """True state on the plane z = zt (array [6, n] float64).

    Along a uniform Bz the longitudinal velocity is constant, so the
    transverse path to the plane is (zt - z) tan(theta); the transverse motion
    is integrated numerically over that path."""
    x, y, z, k, phi, th = truth
    S = (zt - z) * np.tan(th)
    kappa = curvature_rate(q, k, bz)
    xs, ys, tx, ty = rk4_transverse(x, y, np.cos(phi), np.sin(phi), kappa, S / steps, steps)
    out = np.stack([xs, ys, np.broadcast_to(np.asarray(zt, dtype=np.float64), x.shape).copy(),
                    k, np.arctan2(ty, tx), th])
    return out, S


def simulate_to_r(truth: np.ndarray, q, bz: float, R, h: float = 1.0,
                  s_max: Optional[float] = None, refine: int = 8):
    """True state at the first outward crossing of radius R (float64 [6, n]).

    Fixed RK4 steps of size h until r >= R, then Newton iterations on the
    length f of the last (partial) RK4 step, solving |P(f)|^2 = R^2 with the
    direction returned by the same sub-step as derivative.  Tracks that start
    outside the cylinder or do not reach it within s_max (default 4R) are
    returned as NaN with reached = False."""
    x0, y0, z0, k, phi, th = [np.asarray(a, dtype=np.float64) for a in truth]
    n = x0.shape[0]
    Rv = np.broadcast_to(np.asarray(R, dtype=np.float64), (n,))
    if s_max is None:
        s_max = 4.0 * float(Rv.max()) if n else 0.0
    kappa = np.broadcast_to(curvature_rate(q, k, bz), (n,)).copy()
    X, Y = x0.copy(), y0.copy()
    TX, TY = np.cos(phi), np.sin(phi)
    S = np.zeros(n)
    out_x = np.full(n, np.nan)
    out_y = np.full(n, np.nan)
    out_tx = np.full(n, np.nan)
    out_ty = np.full(n, np.nan)
    out_s = np.full(n, np.nan)
    R2all = Rv * Rv
    active = np.nonzero(X * X + Y * Y < R2all)[0]
    nsteps = int(math.ceil(s_max / h))
    for _ in range(nsteps):
        if active.size == 0:
            break
        xa, ya, txa, tya, ka = X[active], Y[active], TX[active], TY[active], kappa[active]
        R2 = R2all[active]
        xn, yn, txn, tyn = rk4_transverse(xa, ya, txa, tya, ka, h, 1)
        crossed = xn * xn + yn * yn >= R2
        if np.any(crossed):
            c = np.nonzero(crossed)[0]
            xc, yc, txc, tyc, kc, R2c = xa[c], ya[c], txa[c], tya[c], ka[c], R2[c]
            # start from the straight-line estimate inside the step
            b = xc * txc + yc * tyc
            f = np.clip(-b + np.sqrt(np.maximum(b * b - (xc * xc + yc * yc - R2c), 0.0)), 0.0, h)
            for _it in range(refine):
                xf, yf, txf, tyf = rk4_transverse(xc, yc, txc, tyc, kc, f, 1)
                g = xf * xf + yf * yf - R2c
                dg = 2.0 * (xf * txf + yf * tyf)
                f = np.clip(f - g / dg, 0.0, h)
            xf, yf, txf, tyf = rk4_transverse(xc, yc, txc, tyc, kc, f, 1)
            idx = active[c]
            out_x[idx], out_y[idx], out_tx[idx], out_ty[idx] = xf, yf, txf, tyf
            out_s[idx] = S[idx] + f
        keep = ~crossed
        ids = active[keep]
        X[ids], Y[ids], TX[ids], TY[ids] = xn[keep], yn[keep], txn[keep], tyn[keep]
        S[ids] += h
        active = ids
    reached = np.isfinite(out_s)
    cot = np.cos(th) / np.sin(th)
    out = np.stack([out_x, out_y, z0 + out_s * cot, np.where(reached, k, np.nan),
                    np.arctan2(out_ty, out_tx), np.where(reached, th, np.nan)])
    return out, out_s, reached


# --------------------------------------------------------------- generation

def make_covariances(rng: np.random.Generator, k: np.ndarray) -> np.ndarray:
    """C = A A^T + diag(sigma^2) with A_ij ~ N(0, (0.1 sigma_i)^2): float64 [n, 6, 6].

    Row-scaling A by sigma_i keeps every entry of C in the units of
    sigma_i sigma_j, so the correlations are O(0.01..0.1) for every pair."""
    n = k.shape[0]
    sig = np.empty((n, 6))
    sig[:, 0], sig[:, 1], sig[:, 2] = COV_SIGMA[0], COV_SIGMA[1], COV_SIGMA[2]
    sig[:, 3] = COV_SIGMA[3] * k
    sig[:, 4], sig[:, 5] = COV_SIGMA[4], COV_SIGMA[5]
    A = rng.standard_normal((n, 6, 6)) * (0.1 * sig)[:, :, None]
    C = np.einsum("nij,nkj->nik", A, A)
    C[:, np.arange(6), np.arange(6)] += sig * sig
    return C


def pack_sym(C: np.ndarray) -> np.ndarray:
    """[n, 6, 6] -> [21, n] packed lower triangle."""
    n = C.shape[0]
    out = np.empty((21, n), dtype=C.dtype)
    for i in range(6):
        for j in range(i + 1):
            out[tri_index(i, j)] = C[:, i, j]
    return out


def unpack_sym(c21: np.ndarray) -> np.ndarray:
    """[21, n] -> [n, 6, 6]."""
    n = c21.shape[1]
    out = np.empty((n, 6, 6), dtype=c21.dtype)
    for i in range(6):
        for j in range(6):
            out[:, i, j] = c21[tri_index(i, j)]
    return out


def _draw_tracks(rng, n, pt_range, eta_range):
    x = rng.normal(0.0, 0.01, n)
    y = rng.normal(0.0, 0.01, n)
    z = rng.normal(0.0, 5.0, n)
    pt = rng.uniform(pt_range[0], pt_range[1], n)
    phi = rng.uniform(-math.pi, math.pi, n)
    eta = rng.uniform(eta_range[0], eta_range[1], n)
    theta = 2.0 * np.arctan(np.exp(-eta))
    q = np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)
    truth = np.stack([x, y, z, 1.0 / pt, phi, theta])
    return truth, q


def _smear(rng, truth, C):
    """Start state = truth + a draw from N(0, C) (Cholesky factor of C)."""
    L = np.linalg.cholesky(C)
    zz = rng.standard_normal((truth.shape[1], 6))
    d = np.einsum("nij,nj->ni", L, zz)
    start = truth + d.T
    start[4] = np.mod(start[4] + math.pi, 2 * math.pi) - math.pi
    return start


def _surface(v):
    """A scalar surface position, or a float32 [n] array of them."""
    if np.ndim(v) == 0:
        return float(v)
    return np.ascontiguousarray(v, dtype=np.float32)


def make_p2z(n: int, seed: int = 1, pt_range=(0.5, 10.0), eta_range=(1.5, 2.5),
             zt: float = 50.0, bz: float = 3.8, hit_sigma: float = 0.01,
             rk4_steps: int = 24) -> Workload:
    """p2z single step: forward tracks to the plane z = zt, hits smeared in x, y."""
    ss = np.random.SeedSequence(seed)
    r_trk, r_cov, r_smear, r_hit = [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(4)]
    truth, q = _draw_tracks(r_trk, n, pt_range, eta_range)
    C = make_covariances(r_cov, truth[3])
    start = _smear(r_smear, truth, C)
    surf_truth, _ = simulate_to_z(truth, q, bz, zt, steps=rk4_steps)
    hit = np.stack([surf_truth[0] + r_hit.normal(0, hit_sigma, n),
                    surf_truth[1] + r_hit.normal(0, hit_sigma, n),
                    np.broadcast_to(np.asarray(zt, dtype=np.float64), (n,))])
    hitcov = np.zeros((6, n))
    hitcov[0] = hitcov[2] = hitcov[5] = hit_sigma ** 2
    return Workload(kind=P2Z, n=n, bz=bz, surf=_surface(zt),
                    state=start.astype(np.float32), cov=pack_sym(C).astype(np.float32),
                    charge=q, hit=hit.astype(np.float32), hitcov=hitcov.astype(np.float32),
                    truth_start=truth, truth_surface=surf_truth,
                    reached=np.isfinite(surf_truth[0]),
                    description=f"p2z n={n} pT~U{pt_range} eta~U{eta_range} z={zt} Bz={bz} seed={seed}")


def make_p2r(nevts: int, ntrks: int, seed: int = 1, pt_range=(0.5, 10.0),
             eta_range=(-1.5, 1.5), R: float = 30.0, bz: float = 3.8,
             rphi_sigma: float = 0.01, z_sigma: float = 0.05, rk4_h: float = 1.0) -> Workload:
    """p2r single step: central tracks to the cylinder r = R; the hit sits on
    the cylinder, smeared along r*phi and z."""
    n = nevts * ntrks
    ss = np.random.SeedSequence(seed)
    r_trk, r_cov, r_smear, r_hit = [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(4)]
    truth, q = _draw_tracks(r_trk, n, pt_range, eta_range)
    C = make_covariances(r_cov, truth[3])
    start = _smear(r_smear, truth, C)
    surf_truth, _, reached = simulate_to_r(truth, q, bz, R, h=rk4_h)
    phic = np.arctan2(surf_truth[1], surf_truth[0])
    phih = np.where(reached, phic + r_hit.normal(0, rphi_sigma, n) / np.asarray(R), 0.0)
    zh = np.where(reached, surf_truth[2] + r_hit.normal(0, z_sigma, n), 0.0)
    Rv = np.broadcast_to(np.asarray(R, dtype=np.float64), (n,))
    hit = np.stack([Rv * np.cos(phih), Rv * np.sin(phih), zh])
    s, c = np.sin(phih), np.cos(phih)
    hitcov = np.zeros((6, n))
    hitcov[0] = rphi_sigma ** 2 * s * s      # xx
    hitcov[1] = -rphi_sigma ** 2 * s * c     # xy
    hitcov[2] = rphi_sigma ** 2 * c * c      # yy
    hitcov[5] = z_sigma ** 2                 # zz
    return Workload(kind=P2R, n=n, bz=bz, surf=_surface(R),
                    state=start.astype(np.float32), cov=pack_sym(C).astype(np.float32),
                    charge=q, hit=hit.astype(np.float32), hitcov=hitcov.astype(np.float32),
                    truth_start=truth, truth_surface=surf_truth, reached=reached,
                    events=nevts,
                    description=(f"p2r {nevts}x{ntrks} pT~U{pt_range} eta~U{eta_range} "
                                 f"R={R} Bz={bz} seed={seed}"))


# ------------------------------------------------------------------ layouts

def aosoa_blocks(n: int, W: int) -> int:
    return (n + W - 1) // W


def to_aosoa(a: np.ndarray, W: int) -> np.ndarray:
    """[C, n] structure-of-arrays -> [nb, C, W] blocks of W tracks (zero padded)."""
    C, n = a.shape
    nb = aosoa_blocks(n, W)
    pad = np.zeros((C, nb * W), dtype=a.dtype)
    pad[:, :n] = a
    return np.ascontiguousarray(pad.reshape(C, nb, W).transpose(1, 0, 2))


def from_aosoa(b: np.ndarray, n: int) -> np.ndarray:
    """[nb, C, W] -> [C, n]."""
    nb, C, W = b.shape
    return np.ascontiguousarray(b.transpose(1, 0, 2).reshape(C, nb * W)[:, :n])


# ------------------------------------------------------- named workloads

def single_step_p2z(seed: int = 1) -> Workload:
    """p2z single step: 8,192 forward tracks to z = 50 cm."""
    return make_p2z(8192, seed=seed)


def single_step_p2r_paper_scale(seed: int = 1) -> Workload:
    """p2r at the paper's scale: 100 events x 9,600 tracks to r = 30 cm."""
    return make_p2r(100, 9600, seed=seed)


def precision_p2z(n: int = 1_000_000, seed: int = 3) -> Workload:
    """Precision study, p2z half: pT extended to 0.2-100 GeV."""
    return make_p2z(n, seed=seed, pt_range=(0.2, 100.0))


def precision_p2r(n: int = 1_000_000, seed: int = 4) -> Workload:
    """Precision study, p2r half: pT extended to 0.2-100 GeV."""
    return make_p2r(100, n // 100, seed=seed, pt_range=(0.2, 100.0))


# ------------------------------------------------------ multi-layer chain

@dataclasses.dataclass
class ChainWorkload:
    n: int
    bz: float
    kinds: np.ndarray              # int32 [L]: P2Z or P2R per layer
    pos: np.ndarray                # float32 [L]: z of the plane / r of the cylinder
    event_sizes: np.ndarray        # int64 [E] tracks per event (tracks are event-major)
    state: np.ndarray              # float32 [6, n]
    cov: np.ndarray                # float32 [21, n]
    charge: np.ndarray             # int8 [n]
    hit: np.ndarray                # float32 [L, 3, n]
    hitcov: np.ndarray             # float32 [L, 6, n]
    truth_pool_layers: np.ndarray  # float64 [L, 6, m] pool's true states per surface (nan: not reached)
    truth_index: np.ndarray        # int64 [n] pool entry of each track
    description: str = ""

    @property
    def L(self) -> int:
        return int(self.kinds.shape[0])

    def truth_layer(self, l: int, idx=None) -> np.ndarray:
        """True states [6, len(idx)] on surface l (NaN where not reached)."""
        ti = self.truth_index if idx is None else self.truth_index[idx]
        return self.truth_pool_layers[l][:, ti]


def chain_layers(n_barrel: int = 8, n_endcap: int = 7, r_range=(4.0, 110.0),
                 z_range=(30.0, 280.0)):
    """Alternating barrel (p2r) and endcap (p2z) layers: r0, z0, r1, z1, ..."""
    rs = np.linspace(r_range[0], r_range[1], n_barrel)
    zs = np.linspace(z_range[0], z_range[1], n_endcap)
    kinds, pos = [], []
    for i in range(max(n_barrel, n_endcap)):
        if i < n_barrel:
            kinds.append(P2R)
            pos.append(rs[i])
        if i < n_endcap:
            kinds.append(P2Z)
            pos.append(zs[i])
    return np.array(kinds, dtype=np.int32), np.array(pos, dtype=np.float32)


def lognormal_event_sizes(rng, events: int, median: float = 5000.0, sigma: float = 1.0,
                          lo: int = 500, hi: int = 40000) -> np.ndarray:
    sizes = np.exp(rng.normal(math.log(median), sigma, events))
    return np.clip(np.rint(sizes), lo, hi).astype(np.int64)


def make_chain(events: int = 256, seed: int = 1, sizes: Optional[np.ndarray] = None,
               pt_range=(0.5, 10.0), eta_range=(1.5, 2.5), bz: float = 3.8,
               kinds: Optional[np.ndarray] = None, pos: Optional[np.ndarray] = None,
               xy_sigma: float = 0.01, rphi_sigma: float = 0.01, z_sigma: float = 0.05,
               pool: int = 65536, rk4_steps: int = 16, rk4_h: float = 1.0) -> ChainWorkload:
    """Events of lognormal track counts run through a layer sequence.

    As in the paper's mini-apps (section 2: a fixed set of track parameters,
    smeared at random for every track), a pool of true tracks is simulated
    through the layers once; every track takes a true track from the pool,
    its own start-state smear N(0, C) and its own hit smear on each surface.
    p2z planes may lie behind the track; a cylinder is taken at the first
    outward crossing from inside.  Where the true track does not reach a
    surface its hit is a placeholder and the truth is NaN."""
    ss = np.random.SeedSequence(seed)
    r_evt, r_trk, r_pick, r_cov, r_smear, r_hit = [np.random.Generator(np.random.PCG64(s))
                                                   for s in ss.spawn(6)]
    if kinds is None or pos is None:
        kinds, pos = chain_layers()
    if sizes is None:
        sizes = lognormal_event_sizes(r_evt, events)
    n = int(sizes.sum())
    m = int(min(pool, n)) if pool else n
    tpool, qpool = _draw_tracks(r_trk, m, pt_range, eta_range)
    L = len(kinds)
    # the pool's true states on every surface
    ptl = np.full((L, 6, m), np.nan)
    cur = tpool.copy()
    alive = np.ones(m, dtype=bool)
    for l in range(L):
        if kinds[l] == P2Z:
            nxt, _ = simulate_to_z(cur, qpool, bz, float(pos[l]), steps=rk4_steps)
            ok = alive & np.isfinite(nxt[0])
        else:
            nxt, _, reached = simulate_to_r(cur, qpool, bz, float(pos[l]), h=rk4_h)
            ok = alive & reached
        ptl[l] = np.where(ok, nxt, np.nan)
        cur = np.where(ok, nxt, cur)
    idx = np.arange(n) % m if n == m else r_pick.integers(0, m, n)
    truth = tpool[:, idx]
    q = qpool[idx]
    C = make_covariances(r_cov, truth[3])
    start = _smear(r_smear, truth, C)
    hit = np.zeros((L, 3, n), dtype=np.float32)
    hitcov = np.zeros((L, 6, n), dtype=np.float32)
    for l in range(L):
        tx, ty, tz = ptl[l, 0][idx], ptl[l, 1][idx], ptl[l, 2][idx]
        ok = np.isfinite(tx)
        if kinds[l] == P2Z:
            hit[l, 0] = np.where(ok, tx + r_hit.normal(0, xy_sigma, n), 0.0)
            hit[l, 1] = np.where(ok, ty + r_hit.normal(0, xy_sigma, n), 0.0)
            hit[l, 2] = pos[l]
            hitcov[l, 0] = hitcov[l, 2] = hitcov[l, 5] = xy_sigma ** 2
        else:
            R = float(pos[l])
            phic = np.arctan2(ty, tx)
            phih = np.where(ok, phic + r_hit.normal(0, rphi_sigma, n) / R, 0.0)
            hit[l, 0], hit[l, 1] = R * np.cos(phih), R * np.sin(phih)
            hit[l, 2] = np.where(ok, tz + r_hit.normal(0, z_sigma, n), 0.0)
            s, c = np.sin(phih), np.cos(phih)
            hitcov[l, 0] = rphi_sigma ** 2 * s * s
            hitcov[l, 1] = -rphi_sigma ** 2 * s * c
            hitcov[l, 2] = rphi_sigma ** 2 * c * c
            hitcov[l, 5] = z_sigma ** 2
    return ChainWorkload(n=n, bz=bz, kinds=np.asarray(kinds, dtype=np.int32),
                         pos=np.asarray(pos, dtype=np.float32), event_sizes=sizes,
                         state=start.astype(np.float32), cov=pack_sym(C).astype(np.float32),
                         charge=q, hit=hit, hitcov=hitcov, truth_pool_layers=ptl,
                         truth_index=idx,
                         description=(f"chain {len(sizes)} events, {n} tracks, {L} layers, "
                                      f"{m} simulated true tracks"))


# --------------------------------------------- compressed covariance format

# Off-diagonal entries (i > j) in packed lower-triangular order:
# 10, 20, 21, 30, 31, 32, 40, ..., 54.
OFFDIAG = [(i, j) for i in range(6) for j in range(i)]


def compress_cov(cov: np.ndarray):
    """[21, n] packed covariance -> (sigma float32 [6, n], rho float16 [15, n]):
    sigma_i = sqrt(C_ii), rho_ij = C_ij / (sigma_i sigma_j) clamped to [-1, 1]
    (0 where a sigma is 0), rounded to nearest in each format."""
    cov = np.asarray(cov, dtype=np.float64)
    diag = np.stack([cov[tri_index(i, i)] for i in range(6)])
    sig = np.sqrt(np.maximum(diag, 0.0)).astype(np.float32)
    s64 = sig.astype(np.float64)
    rho = np.empty((15, cov.shape[1]), dtype=np.float64)
    for k, (i, j) in enumerate(OFFDIAG):
        den = s64[i] * s64[j]
        with np.errstate(divide="ignore", invalid="ignore"):
            r = np.where(den > 0, cov[tri_index(i, j)] / np.where(den > 0, den, 1.0), 0.0)
        rho[k] = np.clip(r, -1.0, 1.0)
    return sig, rho.astype(np.float16)


def rho_to_layout(rho: np.ndarray, width=None) -> np.ndarray:
    """[15, n] FP16 correlations -> the flat rho array of the compressed store.
    Per block of `width` tracks (width None: SoA, one block of n tracks) seven
    rows of pairs, element 2 r + h of row p holding track r's rho_{2p+h}, then
    one row of rho_14: 15 * width values per block."""
    rho = np.asarray(rho, dtype=np.float16)
    blocks = rho[None] if width is None else to_aosoa(rho, width)  # [nb, 15, w]
    nb, _, w = blocks.shape
    pairs = blocks[:, :14].reshape(nb, 7, 2, w).transpose(0, 1, 3, 2).reshape(nb, 14 * w)
    return np.ascontiguousarray(np.concatenate([pairs, blocks[:, 14]], axis=1)).reshape(-1)


def rho_from_layout(flat: np.ndarray, n: int, width=None) -> np.ndarray:
    """Inverse of rho_to_layout: the flat rho array -> [15, n]."""
    w = n if width is None else width
    nb = 1 if width is None else aosoa_blocks(n, width)
    b = np.asarray(flat, dtype=np.float16).reshape(nb, 15 * w)
    pairs = b[:, :14 * w].reshape(nb, 7, w, 2).transpose(0, 1, 3, 2).reshape(nb, 14, w)
    blocks = np.concatenate([pairs, b[:, None, 14 * w:]], axis=1)
    return np.ascontiguousarray(blocks[0]) if width is None else from_aosoa(blocks, n)


def decompress_cov(sig: np.ndarray, rho: np.ndarray) -> np.ndarray:
    """(sigma [6, n], rho [15, n]) -> [21, n] packed covariance in float64."""
    s = np.asarray(sig, dtype=np.float64)
    r = np.asarray(rho, dtype=np.float64)
    out = np.empty((21, s.shape[1]))
    for i in range(6):
        out[tri_index(i, i)] = s[i] * s[i]
    for k, (i, j) in enumerate(OFFDIAG):
        out[tri_index(i, j)] = r[k] * s[i] * s[j]
    return out
