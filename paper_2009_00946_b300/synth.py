"""Seeded synthetic inputs: von Karman phase screens, frozen flow and
Shack-Hartmann slopes with noise.

This module only manufactures inputs.  It holds none of the solver's
arithmetic and is used by the tests, the benchmark and the smoke check to
feed both the CUDA library and the CPU oracle with identical data.

Recipe (the paper gives no atmosphere; Sec. 4.1 only fixes the asterism):
  * screens: periodic FFT screens with the von Karman spectrum
    0.023 r0_l^{-5/3} (f^2 + L0^{-2})^{-11/6}, r0_l = r0 * cn2_l^{-3/5},
    r0 = 0.157 m at 500 nm, L0 = 25 m, sampled at half the layer-grid spacing;
  * frozen flow: layer l moves at v_l ~ U[5, 25] m/s in a direction
    ~ U[0, 2 pi), 500 frames per second;
  * wavefront sensors: the screens are sampled bilinearly along each guide
    star's line of sight at the nodes of a grid twice as fine as the
    subaperture grid (spacing d/2); each fine cell gives an average-difference
    slope and a subaperture slope is the sum of its four fine slopes divided by
    two (a plane a*x + b*y gives exactly a*d, b*d); Gaussian noise of standard
    deviation sigma is added;
  * truth: the screens sampled at the layer-grid nodes at the frame time.

Seeds: PCG64(seed + 1000 l) for the screen of layer l, PCG64(seed + 1000 l + 1)
for its wind, PCG64([seed + 7, frame]) for the noise of a frame.
"""

from __future__ import annotations

import math

import numpy as np

FRAME_RATE = 500.0


def von_karman_screen(N: int, dx: float, r0: float, L0: float, rng) -> np.ndarray:
    fx = np.fft.fftfreq(N, dx)
    f2 = fx[:, None] ** 2 + fx[None, :] ** 2
    psd = 0.023 * r0 ** (-5.0 / 3.0) * (f2 + 1.0 / L0 ** 2) ** (-11.0 / 6.0)
    psd[0, 0] = 0.0
    df = 1.0 / (N * dx)
    cn = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) * np.sqrt(psd) * df
    return np.fft.fft2(cn).real


def structure_function_vk(r: float, r0: float, L0: float, fmax: float = 200.0, nf: int = 400000) -> float:
    """D(r) = 2 int Phi(f) (1 - J0(2 pi f r)) 2 pi f df, by quadrature."""
    from scipy.special import j0
    f = np.linspace(0.0, fmax, nf)[1:]
    phi = 0.023 * r0 ** (-5.0 / 3.0) * (f ** 2 + 1.0 / L0 ** 2) ** (-11.0 / 6.0)
    integrand = phi * (1.0 - j0(2.0 * math.pi * f * r)) * 2.0 * math.pi * f
    return float(2.0 * np.trapezoid(integrand, f))


def _periodic_bilinear(scr: np.ndarray, dx: float, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    N = scr.shape[0]
    u = X / dx
    v = Y / dx
    i0 = np.floor(v).astype(np.int64)
    j0 = np.floor(u).astype(np.int64)
    tv = v - i0
    tu = u - j0
    i0 %= N
    j0 %= N
    i1 = (i0 + 1) % N
    j1 = (j0 + 1) % N
    return ((1 - tv) * (1 - tu) * scr[i0, j0] + (1 - tv) * tu * scr[i0, j1]
            + tv * (1 - tu) * scr[i1, j0] + tv * tu * scr[i1, j1])


class Atmosphere:
    """Frozen-flow layered atmosphere for one configuration."""

    def __init__(self, cfg: dict, seed: int | None = None):
        self.cfg = cfg
        seed = int(cfg.get("seed", 0) if seed is None else seed)
        self.seed = seed
        D = float(cfg["D"])
        r0 = float(cfg["r0"])
        L0 = float(cfg.get("L0", 25.0))
        self.screens, self.dx, self.wind, self.nodes = [], [], [], []
        fit = cfg.get("fit_dirs", [])
        for l, lay in enumerate(cfg["layers"]):
            h = float(lay["height"])
            n = int(lay["n"])
            ext = 0.0
            for w in cfg["wfs"]:
                H = float(w["gs_height"])
                s = 1.0 - h / H if H > 0 else 1.0
                ext = max(ext, 2.0 * (s * D / 2.0 + max(abs(w["theta_x"]), abs(w["theta_y"])) * h))
            for (tx, ty) in fit:
                ext = max(ext, 2.0 * (D / 2.0 + max(abs(tx), abs(ty)) * h))
            step = ext / (n - 1)
            dx = step / 2.0
            N = 1 << int(math.ceil(math.log2(max(256, 4 * (n - 1)))))
            r0l = r0 * float(lay["cn2"]) ** (-3.0 / 5.0)
            scr = von_karman_screen(N, dx, r0l, L0, np.random.Generator(np.random.PCG64(seed + 1000 * l)))
            wr = np.random.Generator(np.random.PCG64(seed + 1000 * l + 1))
            v = wr.uniform(5.0, 25.0)
            ang = wr.uniform(0.0, 2.0 * math.pi)
            self.screens.append(scr)
            self.dx.append(dx)
            self.wind.append((v * math.cos(ang), v * math.sin(ang)))
            self.nodes.append(-ext / 2.0 + np.arange(n) * step)

    def sample(self, l: int, X: np.ndarray, Y: np.ndarray, frame: int) -> np.ndarray:
        t = frame / FRAME_RATE
        vx, vy = self.wind[l]
        return _periodic_bilinear(self.screens[l], self.dx[l], X - vx * t, Y - vy * t)

    def truth_layers(self, frame: int) -> np.ndarray:
        """Screens at the layer-grid nodes, flat (layer-major, row-major)."""
        out = []
        for l in range(len(self.screens)):
            x = self.nodes[l]
            X, Y = np.meshgrid(x, x, indexing="xy")
            out.append(self.sample(l, X, Y, frame).ravel())
        return np.concatenate(out)

    def wavefront(self, g: int, frame: int, refine: int = 2) -> np.ndarray:
        """Wavefront of guide star g at a grid refine-times finer than its subapertures."""
        cfg = self.cfg
        w = cfg["wfs"][g]
        D = float(cfg["D"])
        n = int(w["n_sub"]) * refine
        x = -D / 2.0 + np.arange(n + 1) * (D / n)
        X, Y = np.meshgrid(x, x, indexing="xy")
        H = float(w["gs_height"])
        acc = np.zeros_like(X)
        for l, lay in enumerate(cfg["layers"]):
            h = float(lay["height"])
            s = 1.0 - h / H if H > 0 else 1.0
            acc += self.sample(l, s * X + w["theta_x"] * h, s * Y + w["theta_y"] * h, frame)
        return acc

    def slopes(self, frame: int, noise: bool = True) -> np.ndarray:
        """Flat slope vector: per WFS, x-slopes then y-slopes, row-major (n_s x n_s)."""
        out = []
        rng = np.random.Generator(np.random.PCG64([self.seed + 7, frame]))
        for g, w in enumerate(self.cfg["wfs"]):
            out.append(fine_grid_slopes(self.wavefront(g, frame), int(w["n_sub"])))
        s = np.concatenate(out)
        if noise:
            sig = np.concatenate([np.full(2 * int(w["n_sub"]) ** 2, float(w["sigma"]))
                                  for w in self.cfg["wfs"]])
            s = s + sig * rng.standard_normal(s.size)
        return s


def fine_grid_slopes(phi_fine: np.ndarray, n_sub: int) -> np.ndarray:
    """Sum of the four fine-cell average-difference slopes of each subaperture, / 2."""
    fx = ((phi_fine[:-1, 1:] - phi_fine[:-1, :-1]) + (phi_fine[1:, 1:] - phi_fine[1:, :-1])) / 2.0
    fy = ((phi_fine[1:, :-1] - phi_fine[:-1, :-1]) + (phi_fine[1:, 1:] - phi_fine[:-1, 1:])) / 2.0
    n = n_sub
    sx = fx.reshape(n, 2, n, 2).sum(axis=(1, 3)) / 2.0
    sy = fy.reshape(n, 2, n, 2).sum(axis=(1, 3)) / 2.0
    return np.concatenate([sx.ravel(), sy.ravel()])


def frames(cfg: dict, n_frames: int, noise: bool = True, start: int = 0, seed: int | None = None):
    """(slopes, truth) for frames start..start+n_frames-1 as float64 arrays."""
    atm = Atmosphere(cfg, seed)
    S = np.stack([atm.slopes(start + k, noise) for k in range(n_frames)])
    T = np.stack([atm.truth_layers(start + k) for k in range(n_frames)])
    return S, T


def random_slopes(cfg: dict, seed: int, scale: float = 1.0) -> np.ndarray:
    """White Gaussian slopes (for operator-level checks)."""
    n = sum(2 * int(w["n_sub"]) ** 2 for w in cfg["wfs"])
    return scale * np.random.Generator(np.random.PCG64(seed)).standard_normal(n)


def random_coeffs(cfg: dict, seed: int) -> np.ndarray:
    n = sum(int(l["n"]) ** 2 for l in cfg["layers"])
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(n)
