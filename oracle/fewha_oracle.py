"""FEWHA oracle: a plain, slow, FP64 CPU restatement of the FEWHA hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code,
header, table or constant generator with the CUDA library
(``paper_2009_00946_b300``), and it imports nothing from it.  Inputs (slopes,
configurations) are passed in by the caller.

Paper: B. Stadler, R. Biasi, M. Manetti, R. Ramlau, "Real-time implementation
of an iterative solver for atmospheric tomography", arXiv:2009.00946.

What is computed (paper section / equation / algorithm):
  * Sec. 2.1: subaperture grid, Shack-Hartmann operator Gamma (bilinear FE
    model), NGS/LGS geometric propagation P (cone effect for LGS).
  * Sec. 2.2, Eq. (fewha): M = W^{-T} A^T C^{-1} A W^{-1} + alpha D and
    b = W^{-T} A^T C^{-1} s, with W an orthonormal wavelet transform
    (db3, periodic), so W^{-T} = W (forward) and W^{-1} = W^T (inverse).
  * Alg. 2 ("PCG on GPU"): the single-reduction PCG, and textbook PCG beside it.
  * Alg. 1: RHS, warm restart of the residual, PCG, fitting, open-loop gain;
    closed loop: pseudo-open-loop slopes s + Gamma P_DM a^(-1) and the gain
    a^(1) = a^(0) + gain (a~ - a^(-1)).

Readings taken where the paper is silent or garbled (each one also listed in
the design notes of the repository):
  R1  Grid nodes x_i = -D/2 + i*d, i = 0..n_s, d = D/n_s (Sec. 2.1 prints
      "-D/2 + i"; the (n_s+1)^2 node count of Table 1 needs the factor d).
      Index i is the y (row) axis, j the x (column) axis.
  R2  The second term of s^y (Sec. 2.1) is read as (phi_{i+1,j+1} - phi_{i,j+1}),
      the mirror image of s^x; only that reading annihilates constants.
  R3  Layer grid: n_l x n_l nodes, X_p = -E_l/2 + p*delta_l,
      delta_l = E_l/(n_l - 1), E_l = max over guide stars (and fitting
      directions, NGS-type) and both axes of 2*(s*D/2 + |theta_axis|*h_l),
      s = 1 - h_l/H (1 for NGS).  Bilinear cell = clamp(floor(u), 0, n_l-2).
  R4  Periodic db3 DWT, Mallat layout; each level transforms rows then
      columns of the top-left LL block; synthesis is the exact transpose.
  R5  D_l(j) = r0^{5/3} / (gamma_l * delta_l^{5/3} * 2^{11 j / 3}), j = 1 finest,
      the LL block takes j = J_l (Kolmogorov scaling of wavelet variance).
  R6  C_eta^{-1} = diag(mask_g / sigma_g^2); a subaperture is active when its
      centre lies in the annulus obstruction*D/2 <= r <= D/2.
  R7  Jacobi preconditioner J = diag(M), exactly.
  R8  Alg. 2: exactly n_iter iterations; first iteration beta = 0,
      alpha_0 = rho/mu; p, q are not carried across frames.
  R9  Warm restart (Alg. 1): r = (b1 - b0) + r0, replaced by r = b1 - M c0
      every k_rr frames.
  R10 Fitting for L > M: least squares over the fitting directions,
      min sum_t |P^DM_t a - P^lay_t phi|^2 + eps |a|^2, plain CG, n_fit
      iterations warm-started from the previous solution.
  R14 Low-order sensors (n_sub <= 2, the tip-tilt sensors of Sec. 4.1) have
      every subaperture active.
  R15 LGS tip-tilt (optional, cfg "lgs_tip_tilt_filter"): a laser guide
      star cannot sense tip and tilt, so for an LGS sensor
      C_g^{-1} = w_g (Mk - Mk 1 1^T Mk / n_act) on each slope axis (Mk the
      mask, n_act its active count): the weighted slopes lose their mean over
      the active subapertures.
  R16 L = M with every mirror at its layer's height (Sec. 4.1): the fit is
      the bilinear sampling of layer m at mirror m's actuators (no least
      squares); the layer grid's extent also covers that actuator grid.
  R17 Operating modes of the fit (Sec. 1, Sec. 4.3): MCAO fits every mirror
      over every fitting direction (R10); LTAO is the case of one mirror and
      one direction (the object); MOAO (cfg "fit_mode": "moao") gives each
      fitting direction t its own mirror m = t, fitted in that direction
      alone: min sum_t |P^DM_{t,t} a_t - P^lay_t phi|^2 + eps |a|^2, eps from
      the same diagonal restricted to the pairs (t, t).  MOAO mirrors are not
      seen by the sensors, so MOAO runs open loop.
  R18 Modified Jacobi (Sec. 3.3 names a Jacobi preconditioner with different
      weights for low and high frequencies, after a reference not available
      here): J_i = omega_{j(i)} diag(M)_i, j(i) the DWT level of coefficient i
      (1 = finest, J_l = the LL block), omega_j > 0 from cfg
      "jacobi_level_weights" (a list over j = 1, 2, ...; levels past its end
      take 1).  All omega_j = 1 is the plain Jacobi of R7; the weights
      themselves are parameters, not the paper's.
  R13 Closed loop (Alg. 1): the mirrors' contribution to sensor g is
      Gamma_g sum_m P_{g,m} a_m, P_{g,m} the bilinear mirror m (height h_m)
      sampled at the sensor's nodes as a layer is (shift theta_g h_m, cone
      factor 1 - h_m/H_g); every subaperture, active or not, is added (the
      mask enters only through C^{-1}).

Parity unpinned relative to the paper itself (pinned only by the readings
above, which the CUDA library implements independently): the constant in D,
the preconditioner beyond plain Jacobi, the fitting operator for L > M, the
layer-grid extents and the pupil-mask rule.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ARCSEC = math.pi / (180.0 * 3600.0)
GEOM_TOL = 1e-9


class GeometryError(ValueError):
    """A sample point falls outside a layer (or mirror) grid."""


class BreakdownError(ArithmeticError):
    """The PCG step length denominator is not positive (Alg. 2)."""


# ---------------------------------------------------------------------------
# db3 filters (Sec. 2.2: compactly supported orthonormal wavelets)
# ---------------------------------------------------------------------------

def daubechies_filters(N: int):
    """Daubechies' extremal-phase filter with N vanishing moments.

    Spectral factorisation: |m0(w)|^2 = cos^{2N}(w/2) P(sin^2(w/2)) with
    P(y) = sum_{k<N} C(N-1+k, k) y^k.  With z = e^{-iw},
    sin^2(w/2) = -(z-1)^2/(4z); z^{N-1} P(.) is a polynomial of degree 2N-2
    whose roots come in pairs (r, 1/r); the roots inside the unit circle give
    the extremal-phase factor.  Returns (h, g) with sum h = sqrt(2) and
    g_k = (-1)^k h_{2N-1-k}.
    """
    # polynomial in z (increasing powers), Q(z) = sum_k C(N-1+k,k) (-1)^k (z-1)^{2k} z^{N-1-k} / 4^k
    Q = np.zeros(2 * N - 1)
    for k in range(N):
        ck = math.comb(N - 1 + k, k) * (-1) ** k / 4.0 ** k
        # (z-1)^{2k} coefficients, increasing powers
        zk = np.array([math.comb(2 * k, i) * (-1) ** (2 * k - i) for i in range(2 * k + 1)], dtype=float)
        shift = N - 1 - k
        Q[shift:shift + 2 * k + 1] += ck * zk
    if N > 1:
        roots = np.roots(Q[::-1])
        inside = roots[np.abs(roots) < 1.0]
    else:
        inside = np.array([])
    # m0 ~ (1+z)^N * prod (z - r)  (increasing powers of z)
    poly = np.array([1.0])
    for _ in range(N):
        poly = np.convolve(poly, [1.0, 1.0])
    for r in inside:
        poly = np.convolve(poly, [-r, 1.0])
    h = np.real(poly)
    h = h * (math.sqrt(2.0) / h.sum())
    # extremal phase with the energy at the start: reverse if needed
    if abs(h[0]) < abs(h[-1]):
        h = h[::-1].copy()
    L = h.size
    g = np.array([(-1) ** k * h[L - 1 - k] for k in range(L)])
    return h, g


DB3_H, DB3_G = daubechies_filters(3)


# ---------------------------------------------------------------------------
# periodic 1D / 2D DWT (reading R4)
# ---------------------------------------------------------------------------

def analysis_1d(x: np.ndarray, axis: int, h=None, g=None) -> np.ndarray:
    """One periodic analysis level along ``axis``: [a | d],
    a_k = sum_n h_n x_{(2k+n) mod m}, d_k = sum_n g_n x_{(2k+n) mod m}."""
    h = DB3_H if h is None else h
    g = DB3_G if g is None else g
    x = np.moveaxis(np.asarray(x, dtype=np.float64), axis, 0)
    m = x.shape[0]
    assert m % 2 == 0 and m >= 2
    k = np.arange(m // 2)
    a = np.zeros((m // 2,) + x.shape[1:])
    d = np.zeros((m // 2,) + x.shape[1:])
    for n in range(h.size):
        xs = x[(2 * k + n) % m]
        a += h[n] * xs
        d += g[n] * xs
    return np.moveaxis(np.concatenate([a, d], axis=0), 0, axis)


def synthesis_1d(y: np.ndarray, axis: int, h=None, g=None) -> np.ndarray:
    """Transpose of :func:`analysis_1d`: x_{(2k+n) mod m} += h_n a_k + g_n d_k."""
    h = DB3_H if h is None else h
    g = DB3_G if g is None else g
    y = np.moveaxis(np.asarray(y, dtype=np.float64), axis, 0)
    m = y.shape[0]
    assert m % 2 == 0 and m >= 2
    a, d = y[: m // 2], y[m // 2:]
    k = np.arange(m // 2)
    x = np.zeros_like(y)
    for n in range(h.size):
        idx = (2 * k + n) % m          # injective in k for fixed n
        x[idx] += h[n] * a + g[n] * d
    return np.moveaxis(x, 0, axis)


def fwd_dwt2(layer: np.ndarray, J: int) -> np.ndarray:
    """Forward (analysis) periodic 2D DWT W, J levels, Mallat layout.
    Level j acts on the top-left block of side n/2^{j-1}: rows, then columns."""
    c = np.array(layer, dtype=np.float64, copy=True)
    n = c.shape[0]
    for j in range(1, J + 1):
        m = n >> (j - 1)
        blk = analysis_1d(c[:m, :m], axis=1)
        blk = analysis_1d(blk, axis=0)
        c[:m, :m] = blk
    return c


def inv_dwt2(coeffs: np.ndarray, J: int) -> np.ndarray:
    """Inverse (synthesis) 2D DWT W^{-1} = W^T: the exact transpose of
    :func:`fwd_dwt2`, levels in reverse order, columns then rows."""
    x = np.array(coeffs, dtype=np.float64, copy=True)
    n = x.shape[0]
    for j in range(J, 0, -1):
        m = n >> (j - 1)
        blk = synthesis_1d(x[:m, :m], axis=0)
        blk = synthesis_1d(blk, axis=1)
        x[:m, :m] = blk
    return x


def level_map(n: int, J: int) -> np.ndarray:
    """Level j of each Mallat coefficient (1 = finest; the LL block is J)."""
    i = np.arange(n)
    mx = np.maximum(i[:, None], i[None, :])
    lev = np.full((n, n), J, dtype=np.int64)
    for j in range(J, 0, -1):
        lev[mx >= (n >> j)] = j
    return lev


def level_functions_1d(n: int, j: int) -> np.ndarray:
    """Rows 0..m-1: scaling functions at level j; rows m..2m-1: wavelets at
    level j (m = n/2^j), as vectors on the fine grid of length n."""
    m2 = n >> (j - 1)
    X = synthesis_1d(np.eye(m2), axis=1)
    for _ in range(j - 1, 0, -1):
        X = synthesis_1d(np.concatenate([X, np.zeros_like(X)], axis=1), axis=1)
    return X


# ---------------------------------------------------------------------------
# Shack-Hartmann operator Gamma (Sec. 2.1, reading R2)
# ---------------------------------------------------------------------------

def Gamma(psi: np.ndarray):
    """Average slopes of the bilinear wavefront over each subaperture.
    psi: (n+1, n+1) nodal values [i (y), j (x)].  Returns (sx, sy), (n, n)."""
    sx = ((psi[:-1, 1:] - psi[:-1, :-1]) + (psi[1:, 1:] - psi[1:, :-1])) / 2.0
    sy = ((psi[1:, :-1] - psi[:-1, :-1]) + (psi[1:, 1:] - psi[:-1, 1:])) / 2.0
    return sx, sy


def Gamma_T(sx: np.ndarray, sy: np.ndarray) -> np.ndarray:
    """Transpose of :func:`Gamma`, written as the scatter of its stencil."""
    n = sx.shape[0]
    psi = np.zeros((n + 1, n + 1))
    psi[:-1, 1:] += sx / 2.0
    psi[:-1, :-1] -= sx / 2.0
    psi[1:, 1:] += sx / 2.0
    psi[1:, :-1] -= sx / 2.0
    psi[1:, :-1] += sy / 2.0
    psi[:-1, :-1] -= sy / 2.0
    psi[1:, 1:] += sy / 2.0
    psi[:-1, 1:] -= sy / 2.0
    return psi


def subaperture_mask(n: int, obstruction: float) -> np.ndarray:
    """Reading R6: centre of subaperture (i, j) at ((2j+1-n), (2i+1-n)) * d/2;
    active iff (obstruction*n)^2 <= (2j+1-n)^2 + (2i+1-n)^2 <= n^2.
    Reading R14: a low-order (tip-tilt) sensor, n <= 2, has every
    subaperture active (its subapertures span the whole pupil)."""
    if n <= 2:
        return np.ones((n, n))
    c = 2 * np.arange(n) + 1 - n
    r2 = c[:, None] ** 2 + c[None, :] ** 2
    return ((r2 <= n * n) & (r2 >= (obstruction * n) ** 2)).astype(np.float64)


# ---------------------------------------------------------------------------
# Geometry (Sec. 2.1 grids and propagation, readings R1, R3)
# ---------------------------------------------------------------------------

def _bilinear_table(u: np.ndarray, n: int):
    if np.any(u < -GEOM_TOL) or np.any(u > n - 1 + GEOM_TOL):
        raise GeometryError("sample point outside the grid: u in [%g, %g], grid 0..%d"
                            % (u.min(), u.max(), n - 1))
    cell = np.clip(np.floor(u).astype(np.int64), 0, n - 2)
    return cell, u - cell


def mirror_size(D: float, dirs, h: float, pitch: float) -> tuple:
    """Actuators per side of a mirror at height h that covers the telescope
    footprint in every fitting direction: (n_a, pitch)."""
    half = D / 2.0 + max([max(abs(tx), abs(ty)) for (tx, ty) in dirs] + [0.0]) * h
    return int(math.ceil(2.0 * half / pitch - 1e-9)) + 1, pitch


@dataclass
class Params:
    """Differentiable parameters: Cn^2 fractions gamma_l, alpha, WFS weights w_g."""
    cn2: np.ndarray
    alpha: float
    w: np.ndarray


class Geometry:
    """All derived geometry of one tomography instance, in FP64."""

    def __init__(self, cfg: dict):
        self.cfg = cfg
        self.D = float(cfg["D"])
        self.obstruction = float(cfg.get("obstruction", 0.0))
        self.r0 = float(cfg["r0"])
        self.wfs = cfg["wfs"]
        self.layers = cfg["layers"]
        self.G = len(self.wfs)
        self.L = len(self.layers)
        self.fit_dirs = [tuple(t) for t in cfg.get("fit_dirs", [])]
        self.dms = cfg.get("dms", [])
        self.fit_mode = str(cfg.get("fit_mode", "mcao")).lower()   # R17
        if self.fit_mode not in ("mcao", "moao"):
            raise ValueError("fit_mode must be 'mcao' or 'moao'")
        self.moao = self.fit_mode == "moao"
        if self.moao and len(self.dms) != len(self.fit_dirs):
            raise ValueError("MOAO needs one mirror per fitting direction")

        # WFS grids (R1)
        self.n_sub = [int(w["n_sub"]) for w in self.wfs]
        self.d = [self.D / n for n in self.n_sub]
        self.x_nodes = [-self.D / 2.0 + np.arange(n + 1) * (self.D / n) for n in self.n_sub]
        self.mask = [subaperture_mask(n, self.obstruction) for n in self.n_sub]
        self.nact = [float(m.sum()) for m in self.mask]
        tt = bool(cfg.get("lgs_tip_tilt_filter", False))
        self.tt = [tt and float(w.get("gs_height", 0.0)) > 0.0 for w in self.wfs]

        # co-located mirrors (R16): L = M, mirror m at layer m's height (not
        # for MOAO, whose mirrors each belong to one direction, R17)
        self.colocated = bool(self.dms) and not self.moao and len(self.dms) == self.L and all(
            abs(float(d["height"]) - float(l["height"])) <= 1e-6 * max(1.0, float(l["height"]))
            for d, l in zip(self.dms, self.layers))

        # layer grids (R3)
        self.n = [int(l["n"]) for l in self.layers]
        self.J = [int(l["levels"]) for l in self.layers]
        self.h = [float(l["height"]) for l in self.layers]
        self.E, self.delta, self.X0 = [], [], []
        for l in range(self.L):
            h = self.h[l]
            ext = 0.0
            for g in range(self.G):
                s = self.scale(g, l)
                th = max(abs(self.wfs[g]["theta_x"]), abs(self.wfs[g]["theta_y"]))
                ext = max(ext, 2.0 * (s * self.D / 2.0 + th * h))
            for (tx, ty) in self.fit_dirs:
                ext = max(ext, 2.0 * (self.D / 2.0 + max(abs(tx), abs(ty)) * h))
            if self.colocated:
                na, p = mirror_size(self.D, self.fit_dirs, float(self.dms[l]["height"]), float(self.dms[l]["pitch"]))
                ext = max(ext, (na - 1) * p)
            self.E.append(ext)
            self.delta.append(ext / (self.n[l] - 1))
            self.X0.append(-ext / 2.0)

        # flat coefficient vector: layer-major, row-major within a layer
        self.off = np.concatenate([[0], np.cumsum([n * n for n in self.n])]).astype(np.int64)
        self.N = int(self.off[-1])
        self.soff = np.concatenate([[0], np.cumsum([2 * n * n for n in self.n_sub])]).astype(np.int64)
        self.S = int(self.soff[-1])

        # bilinear sample tables per (g, l): (cy, ty, cx, tx)
        self.tab = [[self._table(g, l) for l in range(self.L)] for g in range(self.G)]

    def scale(self, g: int, l: int) -> float:
        """Cone factor 1 - h_l/H_g for an LGS, 1 for an NGS (Sec. 2.1)."""
        H = float(self.wfs[g].get("gs_height", 0.0))
        return 1.0 - self.h[l] / H if H > 0.0 else 1.0

    def _table(self, g: int, l: int):
        s = self.scale(g, l)
        x = self.x_nodes[g]
        h = self.h[l]
        ux = (s * x + self.wfs[g]["theta_x"] * h - self.X0[l]) / self.delta[l]
        uy = (s * x + self.wfs[g]["theta_y"] * h - self.X0[l]) / self.delta[l]
        cx, tx = _bilinear_table(ux, self.n[l])
        cy, ty = _bilinear_table(uy, self.n[l])
        return cy, ty, cx, tx

    def layer(self, v: np.ndarray, l: int) -> np.ndarray:
        return v[self.off[l]:self.off[l + 1]].reshape(self.n[l], self.n[l])

    def split_slopes(self, s: np.ndarray, g: int):
        n = self.n_sub[g]
        blk = s[self.soff[g]:self.soff[g + 1]].reshape(2, n, n)
        return blk[0], blk[1]

    def default_params(self) -> Params:
        return Params(cn2=np.array([float(l["cn2"]) for l in self.layers]),
                      alpha=float(self.cfg["alpha"]),
                      w=np.array([1.0 / float(w["sigma"]) ** 2 for w in self.wfs]))

    def D_diag(self, params: Params) -> np.ndarray:
        """Reading R5: diagonal regulariser D in the wavelet domain, flat."""
        out = np.empty(self.N)
        for l in range(self.L):
            lev = level_map(self.n[l], self.J[l])
            Dl = self.r0 ** (5.0 / 3.0) / (params.cn2[l] * self.delta[l] ** (5.0 / 3.0)
                                          * 2.0 ** (11.0 * lev / 3.0))
            out[self.off[l]:self.off[l + 1]] = Dl.ravel()
        return out


# ---------------------------------------------------------------------------
# propagation P and its transpose (Sec. 2.1, NGS and LGS)
# ---------------------------------------------------------------------------

def P_layer(geom: Geometry, phi_l: np.ndarray, g: int, l: int) -> np.ndarray:
    """Bilinear interpolation of layer l at the nodes of WFS g (one term of P_g)."""
    cy, ty, cx, tx = geom.tab[g][l]
    Ty, Tx = ty[:, None], tx[None, :]
    return ((1 - Ty) * (1 - Tx) * phi_l[np.ix_(cy, cx)]
            + (1 - Ty) * Tx * phi_l[np.ix_(cy, cx + 1)]
            + Ty * (1 - Tx) * phi_l[np.ix_(cy + 1, cx)]
            + Ty * Tx * phi_l[np.ix_(cy + 1, cx + 1)])


def P_apply(geom: Geometry, phi: list, g: int) -> np.ndarray:
    """psi_g = P_g phi = sum_l phi_l((1 - h_l/H) x + theta_g h_l)."""
    n = geom.n_sub[g]
    psi = np.zeros((n + 1, n + 1))
    for l in range(geom.L):
        psi += P_layer(geom, phi[l], g, l)
    return psi


def PT_layer(geom: Geometry, psi: np.ndarray, g: int, l: int) -> np.ndarray:
    """Transpose of :func:`P_layer`: scatter of the bilinear weights."""
    cy, ty, cx, tx = geom.tab[g][l]
    out = np.zeros((geom.n[l], geom.n[l]))
    CY, CX = np.meshgrid(cy, cx, indexing="ij")
    Ty, Tx = np.meshgrid(ty, tx, indexing="ij")
    np.add.at(out, (CY, CX), (1 - Ty) * (1 - Tx) * psi)
    np.add.at(out, (CY, CX + 1), (1 - Ty) * Tx * psi)
    np.add.at(out, (CY + 1, CX), Ty * (1 - Tx) * psi)
    np.add.at(out, (CY + 1, CX + 1), Ty * Tx * psi)
    return out


# ---------------------------------------------------------------------------
# operator M and right-hand side b (Eq. fewha)
# ---------------------------------------------------------------------------

def layers_from_coeffs(geom: Geometry, c: np.ndarray) -> list:
    """phi = W^{-1} c = W^T c, per layer."""
    return [inv_dwt2(geom.layer(c, l), geom.J[l]) for l in range(geom.L)]


def coeffs_from_layers(geom: Geometry, y: list) -> np.ndarray:
    """W^{-T} y = W y, concatenated."""
    return np.concatenate([fwd_dwt2(y[l], geom.J[l]).ravel() for l in range(geom.L)])


def noise_weight(geom: Geometry, params: Params, g: int, sx: np.ndarray, sy: np.ndarray):
    """C_g^{-1} applied to the slopes of sensor g: w_g mask s, and for a
    tip-tilt-filtered LGS (R15) minus the active-subaperture mean of each axis."""
    mk, w = geom.mask[g], params.w[g]
    if geom.tt[g]:
        sx = sx - float(np.sum(mk * sx)) / geom.nact[g]
        sy = sy - float(np.sum(mk * sy)) / geom.nact[g]
    return w * mk * sx, w * mk * sy


def masked_dot(geom: Geometry, g: int, ax, ay, bx, by) -> float:
    """a^T C_g^{-1} b / w_g for two slope fields of sensor g (R6, R15)."""
    mk = geom.mask[g]
    v = float(np.sum(mk * (ax * bx + ay * by)))
    if geom.tt[g]:
        v -= (float(np.sum(mk * ax)) * float(np.sum(mk * bx)) + float(np.sum(mk * ay)) * float(np.sum(mk * by))) \
            / geom.nact[g]
    return v


def apply_data_term(geom: Geometry, c: np.ndarray, params: Params) -> np.ndarray:
    """W P^T Gamma^T C^{-1} Gamma P W^T c (the first term of M)."""
    phi = layers_from_coeffs(geom, c)
    y = [np.zeros((n, n)) for n in geom.n]
    for g in range(geom.G):
        psi = P_apply(geom, phi, g)
        sx, sy = Gamma(psi)
        psi_p = Gamma_T(*noise_weight(geom, params, g, sx, sy))
        for l in range(geom.L):
            y[l] += PT_layer(geom, psi_p, g, l)
    return coeffs_from_layers(geom, y)


def apply_M(geom: Geometry, c: np.ndarray, params: Params | None = None) -> np.ndarray:
    """M c = (W P^T Gamma^T C^{-1} Gamma P W^T + alpha D) c   (Eq. fewha)."""
    params = geom.default_params() if params is None else params
    return apply_data_term(geom, c, params) + params.alpha * geom.D_diag(params) * c


def rhs(geom: Geometry, s: np.ndarray, params: Params | None = None) -> np.ndarray:
    """b = W P^T Gamma^T C^{-1} s   (Eq. fewha right-hand side; Alg. 1 RHS)."""
    params = geom.default_params() if params is None else params
    y = [np.zeros((n, n)) for n in geom.n]
    for g in range(geom.G):
        sx, sy = geom.split_slopes(s, g)
        psi_p = Gamma_T(*noise_weight(geom, params, g, sx, sy))
        for l in range(geom.L):
            y[l] += PT_layer(geom, psi_p, g, l)
    return coeffs_from_layers(geom, y)


def forward_slopes(geom: Geometry, phi: list) -> np.ndarray:
    """s = A phi = (Gamma_g P_g phi)_g (Eq. atmo), flat slope vector."""
    out = np.empty(geom.S)
    for g in range(geom.G):
        sx, sy = Gamma(P_apply(geom, phi, g))
        out[geom.soff[g]:geom.soff[g + 1]] = np.concatenate([sx.ravel(), sy.ravel()])
    return out


# ---------------------------------------------------------------------------
# Jacobi preconditioner J = diag(M)  (reading R7)
# ---------------------------------------------------------------------------

def _interp_matrix(cell: np.ndarray, t: np.ndarray, n: int) -> np.ndarray:
    Pm = np.zeros((cell.size, n))
    Pm[np.arange(cell.size), cell] += 1 - t
    Pm[np.arange(cell.size), cell + 1] += t
    return Pm


def jacobi_diag(geom: Geometry, params: Params | None = None) -> np.ndarray:
    """diag(M)_i = alpha D_i + sum_g w_g |mask_g Gamma P_g W^T e_i|^2, exactly.

    Each 2D basis function is the tensor product f_y (x) f_x of two 1D level-j
    functions (R4), P_gl is the tensor product of 1D interpolations, and Gamma
    factors into an average in one axis times a difference in the other, so
    |mask Gamma P (f_y (x) f_x)|^2 = (A u)^2 . mask . (D v)^2 + (D u)^2 . mask . (A v)^2
    with u = P_y f_y, v = P_x f_x.  Checked against the diagonal of the densely
    assembled M on small grids.
    """
    params = geom.default_params() if params is None else params
    diag = params.alpha * geom.D_diag(params)
    for l in range(geom.L):
        n, J = geom.n[l], geom.J[l]
        lev = level_map(n, J)
        Y, X = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        acc = np.zeros((n, n))
        for j in range(1, J + 1):
            F = level_functions_1d(n, j)          # (2 m_j, n)
            sel = lev == j
            for g in range(geom.G):
                cy, ty, cx, tx = geom.tab[g][l]
                U = F @ _interp_matrix(cy, ty, n).T   # (2m, n_s+1) along y
                V = F @ _interp_matrix(cx, tx, n).T   # along x
                AU, DU = (U[:, :-1] + U[:, 1:]) / 2.0, U[:, 1:] - U[:, :-1]
                AV, DV = (V[:, :-1] + V[:, 1:]) / 2.0, V[:, 1:] - V[:, :-1]
                mk = geom.mask[g]
                Q = (AU ** 2) @ mk @ (DV ** 2).T + (DU ** 2) @ mk @ (AV ** 2).T
                if geom.tt[g]:   # R15: minus the squared active sums of each slope axis
                    Q = Q - ((AU @ mk @ DV.T) ** 2 + (DU @ mk @ AV.T) ** 2) / geom.nact[g]
                acc[sel] += params.w[g] * Q[Y[sel], X[sel]]
        diag[geom.off[l]:geom.off[l + 1]] += acc.ravel()
    return diag


def level_weights(geom: Geometry) -> np.ndarray:
    """omega_{j(i)} for every coefficient (R18): all ones without weights."""
    w = [float(x) for x in geom.cfg.get("jacobi_level_weights", [])]
    if any(not (x > 0.0) for x in w):
        raise ValueError("jacobi_level_weights must be > 0")
    out = np.ones(geom.N)
    for l in range(geom.L):
        lev = level_map(geom.n[l], geom.J[l]).ravel()
        out[geom.off[l]:geom.off[l + 1]] = [w[j - 1] if j <= len(w) else 1.0 for j in lev]
    return out


def preconditioner_diag(geom: Geometry, params: Params | None = None) -> np.ndarray:
    """The Jacobi preconditioner of Alg. 2: diag(M), level-weighted (R7, R18)."""
    return level_weights(geom) * jacobi_diag(geom, params)


def assemble_M_dense(geom: Geometry, params: Params | None = None) -> np.ndarray:
    """Dense M, one column per unit vector (small grids only)."""
    params = geom.default_params() if params is None else params
    M = np.zeros((geom.N, geom.N))
    for i in range(geom.N):
        e = np.zeros(geom.N)
        e[i] = 1.0
        M[:, i] = apply_M(geom, e, params)
    return M


# ---------------------------------------------------------------------------
# PCG (Alg. 2) and textbook PCG
# ---------------------------------------------------------------------------

def pcg_alg2(Mop, Jinv: np.ndarray, c: np.ndarray, r: np.ndarray, n_iter: int,
             trace: list | None = None):
    """Alg. 2, "PCG on GPU for Mc = b", exactly n_iter iterations (R8).

    z = J^{-1} r; s = M z; rho = (r,z); mu = (s,z); beta = rho/rho_old;
    alpha = rho/(mu - rho beta/alpha_old); p = z + beta p; q = s + beta q;
    c = c + alpha p; r = r - alpha q.
    """
    c = np.array(c, dtype=np.float64, copy=True)
    r = np.array(r, dtype=np.float64, copy=True)
    p = q = None
    rho_old = alpha_old = None
    for k in range(n_iter):
        z = Jinv * r
        s = Mop(z)
        rho = float(r @ z)
        mu = float(s @ z)
        if k == 0:
            beta = 0.0
            denom = mu
        else:
            beta = rho / rho_old
            denom = mu - rho * beta / alpha_old
        if not denom > 0.0:
            raise BreakdownError("PCG denominator %r at iteration %d" % (denom, k))
        alpha_k = rho / denom
        rho_old = rho
        p = z if k == 0 else z + beta * p
        q = s if k == 0 else s + beta * q
        c = c + alpha_k * p
        r = r - alpha_k * q
        alpha_old = alpha_k
        if trace is not None:
            trace.append(dict(k=k, rho=rho, mu=mu, beta=beta, alpha=alpha_k))
    return c, r


def pcg_textbook(Mop, Jinv: np.ndarray, c: np.ndarray, b: np.ndarray, n_iter: int,
                 tol: float = 0.0):
    """Hestenes-Stiefel PCG for M c = b (equal to Alg. 2 in exact arithmetic)."""
    c = np.array(c, dtype=np.float64, copy=True)
    r = b - Mop(c)
    z = Jinv * r
    p = z.copy()
    rz = float(r @ z)
    bn = float(np.linalg.norm(b))
    for _ in range(n_iter):
        if tol > 0.0 and np.linalg.norm(r) <= tol * bn:
            break
        q = Mop(p)
        a = rz / float(p @ q)
        c += a * p
        r -= a * q
        z = Jinv * r
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return c, r


# ---------------------------------------------------------------------------
# mirror fitting (Alg. 1, fitting step; reading R10)
# ---------------------------------------------------------------------------

class FitGeometry:
    """Deformable mirrors (piecewise bilinear, nodes at actuators) and the
    least-squares fit over the fitting directions (NGS-type, no cone)."""

    def __init__(self, geom: Geometry):
        cfg = geom.cfg
        self.geom = geom
        self.dirs = geom.fit_dirs
        self.M = len(geom.dms)
        self.n_pupil = int(cfg.get("fit_n_sub", geom.n_sub[0]))
        self.x = -geom.D / 2.0 + np.arange(self.n_pupil + 1) * (geom.D / self.n_pupil)
        self.na, self.pitch, self.A0, self.hm = [], [], [], []
        for dm in geom.dms:
            h, p = float(dm["height"]), float(dm["pitch"])
            na, _ = mirror_size(geom.D, self.dirs, h, p)
            self.na.append(na)
            self.pitch.append(p)
            self.A0.append(-(na - 1) * p / 2.0)
            self.hm.append(h)
        self.aoff = np.concatenate([[0], np.cumsum([n * n for n in self.na])]).astype(np.int64)
        self.NA = int(self.aoff[-1])
        self.lay_tab = [[self._lay(t, l) for l in range(geom.L)] for t in range(len(self.dirs))]
        self.dm_tab = [[self._dm(t, m) for m in range(self.M)] for t in range(len(self.dirs))]
        diag = np.zeros(self.NA)
        for t in range(len(self.dirs)):
            for m in self.mirrors(t):
                cy, ty, cx, tx = self.dm_tab[t][m]
                wy = np.stack([1 - ty, ty]) ** 2
                wx = np.stack([1 - tx, tx]) ** 2
                blk = np.zeros((self.na[m], self.na[m]))
                for a in range(2):
                    for bb in range(2):
                        CY, CX = np.meshgrid(cy + a, cx + bb, indexing="ij")
                        np.add.at(blk, (CY, CX), np.outer(wy[a], wx[bb]))
                diag[self.aoff[m]:self.aoff[m + 1]] += blk.ravel()
        self.eps = 1e-6 * float(diag.mean())

    def _lay(self, t, l):
        g = self.geom
        tx, ty = self.dirs[t]
        ux = (self.x + tx * g.h[l] - g.X0[l]) / g.delta[l]
        uy = (self.x + ty * g.h[l] - g.X0[l]) / g.delta[l]
        cx, wx = _bilinear_table(ux, g.n[l])
        cy, wy = _bilinear_table(uy, g.n[l])
        return cy, wy, cx, wx

    def _dm(self, t, m):
        tx, ty = self.dirs[t]
        ux = (self.x + tx * self.hm[m] - self.A0[m]) / self.pitch[m]
        uy = (self.x + ty * self.hm[m] - self.A0[m]) / self.pitch[m]
        cx, wx = _bilinear_table(ux, self.na[m])
        cy, wy = _bilinear_table(uy, self.na[m])
        return cy, wy, cx, wx

    @staticmethod
    def _interp(grid, tab):
        cy, ty, cx, tx = tab
        Ty, Tx = ty[:, None], tx[None, :]
        return ((1 - Ty) * (1 - Tx) * grid[np.ix_(cy, cx)] + (1 - Ty) * Tx * grid[np.ix_(cy, cx + 1)]
                + Ty * (1 - Tx) * grid[np.ix_(cy + 1, cx)] + Ty * Tx * grid[np.ix_(cy + 1, cx + 1)])

    @staticmethod
    def _interp_T(v, tab, n):
        cy, ty, cx, tx = tab
        out = np.zeros((n, n))
        CY, CX = np.meshgrid(cy, cx, indexing="ij")
        Ty, Tx = np.meshgrid(ty, tx, indexing="ij")
        np.add.at(out, (CY, CX), (1 - Ty) * (1 - Tx) * v)
        np.add.at(out, (CY, CX + 1), (1 - Ty) * Tx * v)
        np.add.at(out, (CY + 1, CX), Ty * (1 - Tx) * v)
        np.add.at(out, (CY + 1, CX + 1), Ty * Tx * v)
        return out

    def dm(self, a, m):
        return a[self.aoff[m]:self.aoff[m + 1]].reshape(self.na[m], self.na[m])

    def mirrors(self, t):
        """Mirrors fitted in direction t: all (MCAO, LTAO) or mirror t (MOAO, R17)."""
        return [t] if self.geom.moao else list(range(self.M))

    def P_dm(self, a, t):
        return sum(self._interp(self.dm(a, m), self.dm_tab[t][m]) for m in self.mirrors(t))

    def P_dm_T(self, v, t):
        ms = self.mirrors(t)
        return np.concatenate([self._interp_T(v, self.dm_tab[t][m], self.na[m]).ravel() if m in ms
                               else np.zeros(self.na[m] * self.na[m]) for m in range(self.M)])

    def colocated_fit(self, phi):
        """R16: mirror m's actuators take layer m's bilinear value at their
        positions (the layer and the mirror share a height)."""
        geom = self.geom
        out = []
        for m in range(self.M):
            X = self.A0[m] + np.arange(self.na[m]) * self.pitch[m]
            c, t = _bilinear_table((X - geom.X0[m]) / geom.delta[m], geom.n[m])
            out.append(self._interp(phi[m], (c, t, c, t)).ravel())
        return np.concatenate(out)

    def wfs_table(self, g: int, m: int):
        """Bilinear sample table of mirror m at the nodes of sensor g (R13)."""
        geom = self.geom
        w = geom.wfs[g]
        H = float(w.get("gs_height", 0.0))
        h = self.hm[m]
        sc = 1.0 - h / H if H > 0.0 else 1.0
        x = geom.x_nodes[g]
        ux = (sc * x + w["theta_x"] * h - self.A0[m]) / self.pitch[m]
        uy = (sc * x + w["theta_y"] * h - self.A0[m]) / self.pitch[m]
        cx, tx = _bilinear_table(ux, self.na[m])
        cy, ty = _bilinear_table(uy, self.na[m])
        return cy, ty, cx, tx

    def dm_to_wfs(self, a, g: int):
        """Nodal field sum_m P_{g,m} a_m of the mirrors seen by sensor g."""
        return sum(self._interp(self.dm(a, m), self.wfs_table(g, m)) for m in range(self.M))

    def dm_slopes(self, a):
        """Gamma_g sum_m P_{g,m} a_m for every sensor: the measurements the
        mirrors' shapes add (Alg. 1, closed loop), flat slope vector."""
        geom = self.geom
        out = np.empty(geom.S)
        for g in range(geom.G):
            sx, sy = Gamma(self.dm_to_wfs(a, g))
            out[geom.soff[g]:geom.soff[g + 1]] = np.concatenate([sx.ravel(), sy.ravel()])
        return out

    def P_lay(self, phi, t):
        return sum(self._interp(phi[l], self.lay_tab[t][l]) for l in range(self.geom.L))

    def normal_op(self, a):
        """(sum_t P_DM_t^T P_DM_t + eps I) a."""
        out = self.eps * a
        for t in range(len(self.dirs)):
            out = out + self.P_dm_T(self.P_dm(a, t), t)
        return out

    def normal_rhs(self, phi):
        out = np.zeros(self.NA)
        for t in range(len(self.dirs)):
            out += self.P_dm_T(self.P_lay(phi, t), t)
        return out

    def fit(self, phi, a0, n_fit):
        """Plain CG on the normal equations, n_fit iterations from a0."""
        x = np.array(a0, dtype=np.float64, copy=True)
        r = self.normal_rhs(phi) - self.normal_op(x)
        p = r.copy()
        rr = float(r @ r)
        for _ in range(n_fit):
            if rr == 0.0:
                break
            q = self.normal_op(p)
            pq = float(p @ q)
            if not pq > 0.0:
                break
            a = rr / pq
            x += a * p
            r -= a * q
            rr_new = float(r @ r)
            p = r + (rr_new / rr) * p
            rr = rr_new
        return x


# ---------------------------------------------------------------------------
# Alg. 1: one reconstruction frame (open loop)
# ---------------------------------------------------------------------------

@dataclass
class FrameState:
    """Alg. 1 inputs carried across frames: c0, b0, r0, a(-1), a(0)."""
    c: np.ndarray
    b: np.ndarray
    r: np.ndarray
    a_prev: np.ndarray | None = None
    a_cur: np.ndarray | None = None
    a_fit: np.ndarray | None = None
    count: int = 0
    extra: dict = field(default_factory=dict)


class Reconstructor:
    """Alg. 1 around Alg. 2 for one geometry; FP64 throughout."""

    def __init__(self, cfg: dict, params: Params | None = None):
        self.geom = Geometry(cfg)
        self.params = self.geom.default_params() if params is None else params
        self.Jdiag = preconditioner_diag(self.geom, self.params)
        self.Jinv = 1.0 / self.Jdiag
        self.fitgeom = FitGeometry(self.geom) if self.geom.dms else None
        self.reset()

    def reset(self):
        N = self.geom.N
        NA = self.fitgeom.NA if self.fitgeom else 0
        self.state = FrameState(c=np.zeros(N), b=np.zeros(N), r=np.zeros(N),
                                a_prev=np.zeros(NA), a_cur=np.zeros(NA), a_fit=np.zeros(NA))

    def Mop(self, v):
        return apply_M(self.geom, v, self.params)

    def frame(self, s: np.ndarray, n_iter: int, warm: bool = True, k_rr: int = 10,
              gain: float = 1.0, n_fit: int = 8, loop: str = "open"):
        """Closed loop: s = s + Gamma P_DM a^(-1) first.  b1 = W P^T Gamma^T
        C^{-1} s; r = (b1 - b0) + r0 (or b1 - M c0 every k_rr frames);
        (c1, r1) = PCG(c0, r); a~ = F W^{-1} c1; open-loop gain
        a1 = (1 - gain) a0 + gain a~, or closed-loop a1 = a0 + gain (a~ - a^(-1))."""
        st = self.state
        if loop not in ("open", "closed"):
            raise ValueError("loop must be 'open' or 'closed'")
        if loop == "closed":
            if self.fitgeom is None:
                raise ValueError("closed loop needs deformable mirrors")
            if self.geom.moao:
                raise ValueError("MOAO mirrors are not seen by the sensors: open loop only (R17)")
            s = s + self.fitgeom.dm_slopes(st.a_prev)
        b1 = rhs(self.geom, s, self.params)
        if not warm:
            c0 = np.zeros(self.geom.N)
            r = b1.copy()
        else:
            c0 = st.c
            if k_rr > 0 and st.count > 0 and st.count % k_rr == 0:
                r = b1 - self.Mop(c0)
            else:
                r = (b1 - st.b) + st.r
        c1, r1 = pcg_alg2(self.Mop, self.Jinv, c0, r, n_iter)
        st.c, st.b, st.r = c1, b1, r1
        st.count += 1
        out = {"c": c1, "b": b1, "r": r1}
        if self.fitgeom is not None:
            phi = layers_from_coeffs(self.geom, c1)
            if self.geom.colocated:
                a_fit = self.fitgeom.colocated_fit(phi)
            else:
                a_fit = self.fitgeom.fit(phi, st.a_fit, n_fit)
            if loop == "closed":
                a_new = st.a_cur + gain * (a_fit - st.a_prev)
            else:
                a_new = (1.0 - gain) * st.a_cur + gain * a_fit
            st.a_prev, st.a_cur, st.a_fit = st.a_cur, a_new, a_fit
            out["a"] = a_new
        return out

    def layers(self, c: np.ndarray | None = None) -> np.ndarray:
        c = self.state.c if c is None else c
        return np.concatenate([p.ravel() for p in layers_from_coeffs(self.geom, c)])


# ---------------------------------------------------------------------------
# reverse mode through the unrolled Alg. 2 (differentiation of the solve)
# ---------------------------------------------------------------------------
# Reading R12: the derivative is taken of the fixed-iteration solve exactly as
# computed (K iterations of Alg. 2 from c = 0, r = b), with the preconditioner
# J held fixed; theta = (Cn^2 fractions gamma_l, alpha, sensor weights w_g).
# M depends on theta through alpha D (D ~ 1/gamma_l) and w_g; b through w_g.

def pcg_alg2_tape(Mop, Jinv: np.ndarray, b: np.ndarray, n_iter: int):
    """Alg. 2 from c = 0, r = b, keeping every intermediate for the adjoint."""
    N = b.size
    c = np.zeros(N)
    r = b.copy()
    p = q = np.zeros(N)
    tape = []
    rho_old = alpha_old = None
    for k in range(n_iter):
        z = Jinv * r
        s = Mop(z)
        rho = float(r @ z)
        mu = float(s @ z)
        if k == 0:
            beta, d = 0.0, mu
        else:
            beta = rho / rho_old
            d = mu - rho * beta / alpha_old
        if not d > 0.0:
            raise BreakdownError("PCG denominator %r at iteration %d" % (d, k))
        alpha = rho / d
        tape.append(dict(r=r, z=z, s=s, p_old=p, q_old=q, rho=rho, mu=mu, beta=beta, d=d, alpha=alpha,
                         rho_old=rho_old, alpha_old=alpha_old))
        p = z + beta * p
        q = s + beta * q
        c = c + alpha * p
        r = r - alpha * q
        tape[-1]["p"] = p
        tape[-1]["q"] = q
        rho_old, alpha_old = rho, alpha
    return c, r, tape


def pcg_alg2_adjoint(Mop, Jinv: np.ndarray, tape: list, cbar: np.ndarray):
    """Adjoint of :func:`pcg_alg2_tape` for a cotangent cbar of the final c.
    Returns (bbar, [(z_k, sbar_k)]): the cotangent of b and, per iteration,
    the pair that contracts with dM/dtheta (s_k = M z_k)."""
    N = cbar.size
    cb = cbar.copy()          # cotangent of c_{k+1}
    rb = np.zeros(N)          # cotangent of r_{k+1}
    pb = np.zeros(N)          # cotangent of p_k (from later iterations)
    qb = np.zeros(N)
    rhob_next = 0.0           # contribution to rho_k from iteration k+1
    alphab_next = 0.0         # contribution to alpha_k from iteration k+1
    pairs = []
    for k in range(len(tape) - 1, -1, -1):
        t = tape[k]
        # c_{k+1} = c_k + alpha_k p_k ; r_{k+1} = r_k - alpha_k q_k
        alphab = alphab_next + float(cb @ t["p"]) - float(rb @ t["q"])
        pb = pb + t["alpha"] * cb
        qb = qb - t["alpha"] * rb
        # p_k = z_k + beta_k p_{k-1} ; q_k = s_k + beta_k q_{k-1}
        zb = pb.copy()
        sb = qb.copy()
        betab = float(pb @ t["p_old"]) + float(qb @ t["q_old"]) if k > 0 else 0.0
        pb_prev = t["beta"] * pb
        qb_prev = t["beta"] * qb
        # alpha_k = rho_k / d_k
        rhob = rhob_next + alphab / t["d"]
        db = -alphab * t["rho"] / t["d"] ** 2
        mub = db
        alphab_prev = 0.0
        rhob_prev = 0.0
        if k > 0:
            # d_k = mu_k - rho_k beta_k / alpha_{k-1}
            rhob -= db * t["beta"] / t["alpha_old"]
            betab -= db * t["rho"] / t["alpha_old"]
            alphab_prev = db * t["rho"] * t["beta"] / t["alpha_old"] ** 2
            # beta_k = rho_k / rho_{k-1}
            rhob += betab / t["rho_old"]
            rhob_prev = -betab * t["rho"] / t["rho_old"] ** 2
        # mu_k = (s_k, z_k) ; rho_k = (r_k, z_k)
        sb = sb + mub * t["z"]
        zb = zb + mub * t["s"] + rhob * t["r"]
        rb_k = rb + rhob * t["z"]
        # s_k = M z_k (M symmetric)
        zb = zb + Mop(sb)
        pairs.append((t["z"], sb))
        # z_k = J^{-1} r_k
        rb = rb_k + Jinv * zb
        pb, qb = pb_prev, qb_prev
        rhob_next, alphab_next = rhob_prev, alphab_prev
        # c_k receives cb unchanged (c_{k+1} = c_k + ...)
    return rb, pairs[::-1]


def _sensor_slopes_of(geom: Geometry, c: np.ndarray):
    """Gamma P_g W^T c for every sensor g: list of (sx, sy)."""
    phi = layers_from_coeffs(geom, c)
    return [Gamma(P_apply(geom, phi, g)) for g in range(geom.G)]


def dM_contract(geom: Geometry, params: Params, z: np.ndarray, sbar: np.ndarray):
    """sbar^T (dM/dtheta) z for theta = (gamma_l..., alpha, w_g...)."""
    D = geom.D_diag(params) / 1.0               # D without alpha
    t = sbar * D * z
    galpha = float(t.sum())
    ggam = np.array([-params.alpha * float(t[geom.off[l]:geom.off[l + 1]].sum()) / params.cn2[l]
                     for l in range(geom.L)])
    A = _sensor_slopes_of(geom, z)
    B = _sensor_slopes_of(geom, sbar)
    gw = np.array([masked_dot(geom, g, A[g][0], A[g][1], B[g][0], B[g][1]) for g in range(geom.G)])
    return ggam, galpha, gw


def db_contract(geom: Geometry, s: np.ndarray, bbar: np.ndarray):
    """bbar^T (db/dw_g) = (Gamma P_g W^T bbar) . (mask_g s_g)."""
    B = _sensor_slopes_of(geom, bbar)
    out = []
    for g in range(geom.G):
        sx, sy = geom.split_slopes(s, g)
        out.append(masked_dot(geom, g, B[g][0], B[g][1], sx, sy))
    return np.array(out)


def slopes_contract(geom: Geometry, params: Params, bbar: np.ndarray) -> np.ndarray:
    """d loss / d s from the cotangent bbar of b: b = W P^T Gamma^T C^{-1} s
    (Eq. (fewha)) is linear in s, so the slope gradient is its transpose
    applied to bbar, C^{-1} Gamma P W^T bbar (C^{-1} symmetric), in the slope
    layout of the measurement vector."""
    B = _sensor_slopes_of(geom, bbar)
    out = []
    for g in range(geom.G):
        wx, wy = noise_weight(geom, params, g, B[g][0], B[g][1])
        out.append(np.concatenate([wx.ravel(), wy.ravel()]))
    return np.concatenate(out)


def solve_loss(geom: Geometry, params: Params, Jinv: np.ndarray, s: np.ndarray, phi_true: np.ndarray,
               n_iter: int):
    """Loss |W^T c_K - phi_true|^2 of one frame solved from a cold start."""
    b = rhs(geom, s, params)
    c, _, _ = pcg_alg2_tape(lambda v: apply_M(geom, v, params), Jinv, b, n_iter)
    phi = np.concatenate([p.ravel() for p in layers_from_coeffs(geom, c)])
    return float(np.sum((phi - phi_true) ** 2))


def solve_loss_grad(geom: Geometry, params: Params, Jinv: np.ndarray, s: np.ndarray, phi_true: np.ndarray,
                    n_iter: int, with_slopes: bool = False):
    """(loss, d loss / d gamma, d loss / d alpha, d loss / d w) by reverse mode;
    with_slopes: also d loss / d s (a fifth entry)."""
    Mop = lambda v: apply_M(geom, v, params)
    b = rhs(geom, s, params)
    c, _, tape = pcg_alg2_tape(Mop, Jinv, b, n_iter)
    phi_l = layers_from_coeffs(geom, c)
    phi = np.concatenate([p.ravel() for p in phi_l])
    res = phi - phi_true
    loss = float(np.sum(res ** 2))
    # phi = W^T c  ->  cbar = W (2 res)
    cbar = coeffs_from_layers(geom, [2.0 * geom.layer(res, l) for l in range(geom.L)])
    bbar, pairs = pcg_alg2_adjoint(Mop, Jinv, tape, cbar)
    ggam = np.zeros(geom.L)
    galpha = 0.0
    gw = np.zeros(geom.G)
    for z, sb in pairs:
        a, b2, c2 = dM_contract(geom, params, z, sb)
        ggam += a
        galpha += b2
        gw += c2
    gw += db_contract(geom, s, bbar)
    if with_slopes:
        return loss, ggam, galpha, gw, slopes_contract(geom, params, bbar)
    return loss, ggam, galpha, gw
