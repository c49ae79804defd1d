// Host-side setup of a FEWHA instance: grids, bilinear sample and gather
// tables, the wavelet-domain regulariser D and the Jacobi diagonal diag(M).
// Everything here runs once per fewha_create, in FP64; the per-frame work
// runs in the CUDA kernels.
#include "setup.h"

#include <algorithm>
#include <cmath>
#include <cstdio>

namespace fewha {

namespace {

constexpr double kGeomTol = 1e-9;

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Bilinear cell and weight of a sample coordinate u (in grid units) on a grid
// with n nodes: cell = clamp(floor(u), 0, n-2), t = u - cell.
bool bilinear_cell(double u, int n, int& cell, double& t) {
    if (!(u >= -kGeomTol) || !(u <= (n - 1) + kGeomTol)) return false;
    int c = (int)std::floor(u);
    c = std::max(0, std::min(c, n - 2));
    cell = c;
    t = u - c;
    return true;
}

// Sample table of the sensor grid (n_sub+1 nodes at spacing D/n_sub, centred)
// on a grid X0 + p*delta (n nodes), for the affine map x -> s*x + th*h.
bool sample_table(double D, int n_sub, double s, double th, double h, double X0, double delta, int n,
                  std::vector<int>& cell, std::vector<double>& t) {
    for (int k = 0; k <= n_sub; ++k) {
        double x = -D / 2.0 + k * (D / n_sub);
        double u = (s * x + th * h - X0) / delta;
        int c;
        double w;
        if (!bilinear_cell(u, n, c, w)) return false;
        cell.push_back(c);
        t.push_back(w);
    }
    return true;
}

// Gather ranges of the transpose: for every grid index q, the contiguous range
// of sample indices k with cell_k in {q-1, q} (cells are non-decreasing in k).
void gather_ranges(const int* cell, int count, int n, std::vector<int>& lo, std::vector<int>& hi) {
    for (int q = 0; q < n; ++q) {
        int a = count, b = 0;
        for (int k = 0; k < count; ++k) {
            if (cell[k] == q - 1 || cell[k] == q) {
                a = std::min(a, k);
                b = std::max(b, k + 1);
            }
        }
        if (a >= b) { a = 0; b = 0; }
        lo.push_back(a);
        hi.push_back(b);
    }
}

// One periodic synthesis level along a vector of even length m (transpose of
// a_k = sum_n h_n x_{2k+n}, d_k = sum_n g_n x_{2k+n}).
void synth1d(const double* y, double* x, int m, const double* h, const double* g) {
    for (int i = 0; i < m; ++i) x[i] = 0.0;
    int half = m / 2;
    for (int k = 0; k < half; ++k)
        for (int n = 0; n < 6; ++n) {
            int i = (2 * k + n) % m;
            x[i] += h[n] * y[k] + g[n] * y[half + k];
        }
}

// Level-j 1D functions on a grid of n: rows 0..m-1 scaling, m..2m-1 wavelets
// (m = n >> j), stored row-major (2m x n).
std::vector<double> level_functions(int n, int j, const double* h, const double* g) {
    int m2 = n >> (j - 1);
    std::vector<double> F((size_t)m2 * n, 0.0);
    std::vector<double> a(n), b(n);
    for (int k = 0; k < m2; ++k) {
        std::fill(a.begin(), a.end(), 0.0);
        a[k] = 1.0;
        int len = m2;
        synth1d(a.data(), b.data(), len, h, g);
        while (len < n) {
            // the current vector is the scaling part of the next finer level
            for (int i = 0; i < len; ++i) a[i] = b[i];
            for (int i = len; i < 2 * len; ++i) a[i] = 0.0;
            len *= 2;
            synth1d(a.data(), b.data(), len, h, g);
        }
        for (int i = 0; i < n; ++i) F[(size_t)k * n + i] = b[i];
    }
    return F;
}

int level_of(int y, int x, int n, int J) {
    int mx = std::max(y, x);
    for (int j = 1; j <= J; ++j)
        if (mx >= (n >> j)) return j;
    return J;
}

}  // namespace

void db3_taps(double h[6], double g[6]) {
    // Daubechies' 6-tap extremal-phase filter in radicals.
    const double r10 = std::sqrt(10.0);
    const double s = std::sqrt(5.0 + 2.0 * r10);
    const double k = 1.0 / (16.0 * std::sqrt(2.0));
    h[0] = (1.0 + r10 + s) * k;
    h[1] = (5.0 + r10 + 3.0 * s) * k;
    h[2] = (10.0 - 2.0 * r10 + 2.0 * s) * k;
    h[3] = (10.0 - 2.0 * r10 - 2.0 * s) * k;
    h[4] = (5.0 + r10 - 3.0 * s) * k;
    h[5] = (1.0 + r10 - s) * k;
    for (int i = 0; i < 6; ++i) g[i] = ((i & 1) ? -1.0 : 1.0) * h[5 - i];
}

// Actuators per side of a mirror at height h covering the telescope
// footprint in every fitting direction (|theta| <= thmax).
static int mirror_actuators(double D, double thmax, double h, double pitch) {
    const double half = D / 2.0 + thmax * h;
    return (int)std::ceil(2.0 * half / pitch - 1e-9) + 1;
}

double reg_diag(double r0, double cn2, double delta, int j) {
    return std::pow(r0, 5.0 / 3.0) / (cn2 * std::pow(delta, 5.0 / 3.0) * std::pow(2.0, 11.0 * j / 3.0));
}

int build_setup(const fewha_geometry& geo, const fewha_profile& prof, HostSetup& o, std::string& err) {
    char buf[256];
    auto fail = [&](int code, const char* msg) {
        err = msg;
        return code;
    };
    if (!(geo.D > 0)) return fail(FEWHA_ERR_ARG, "D must be > 0");
    if (!(geo.obstruction >= 0 && geo.obstruction < 1)) return fail(FEWHA_ERR_ARG, "obstruction must be in [0, 1)");
    if (geo.n_wfs < 1 || geo.n_wfs > FEWHA_MAX_WFS) return fail(FEWHA_ERR_ARG, "n_wfs out of range");
    if (prof.n_layers < 1 || prof.n_layers > FEWHA_MAX_LAYERS) return fail(FEWHA_ERR_ARG, "n_layers out of range");
    if (geo.precision != FEWHA_FP32 && geo.precision != FEWHA_FP64) return fail(FEWHA_ERR_ARG, "precision must be FP32 or FP64");
    if (!(prof.alpha > 0) || !(prof.r0 > 0)) return fail(FEWHA_ERR_ARG, "alpha and r0 must be > 0");
    for (int j = 0; j < FEWHA_MAX_JACOBI_LEVELS; ++j)
        if (!(prof.jacobi_level_weight[j] >= 0.0))
            return fail(FEWHA_ERR_ARG, "jacobi_level_weight must be >= 0 (0: unweighted)");
    if (geo.n_dm < 0 || geo.n_dm > FEWHA_MAX_DMS) return fail(FEWHA_ERR_ARG, "n_dm out of range");
    if (geo.n_fit_dir < 0 || geo.n_fit_dir > FEWHA_MAX_FIT_DIRS) return fail(FEWHA_ERR_ARG, "n_fit_dir out of range");
    if (geo.n_dm > 0 && geo.n_fit_dir < 1) return fail(FEWHA_ERR_ARG, "mirrors need at least one fitting direction");
    if (geo.fit_mode != FEWHA_FIT_MCAO && geo.fit_mode != FEWHA_FIT_MOAO)
        return fail(FEWHA_ERR_ARG, "fit_mode must be FEWHA_FIT_MCAO or FEWHA_FIT_MOAO");
    if (geo.fit_mode == FEWHA_FIT_MOAO && geo.n_dm != geo.n_fit_dir)
        return fail(FEWHA_ERR_ARG, "MOAO needs one mirror per fitting direction");

    o.prec = geo.precision;
    o.D = geo.D;
    o.obstruction = geo.obstruction;
    o.r0 = prof.r0;
    o.alpha = prof.alpha;
    o.L = prof.n_layers;
    o.G = geo.n_wfs;
    o.M = geo.n_dm;
    o.T = geo.n_fit_dir;
    o.moao = geo.fit_mode == FEWHA_FIT_MOAO;
    db3_taps(o.h, o.g);

    // sensors
    o.wfs.resize(o.G);
    long soff = 0, noff = 0, moff = 0;
    for (int g = 0; g < o.G; ++g) {
        HostWfs& w = o.wfs[g];
        w.n = geo.n_sub[g];
        if (w.n < 1 || w.n > 1024) return fail(FEWHA_ERR_ARG, "n_sub out of range (1..1024)");
        if (!(geo.noise_sigma[g] > 0)) return fail(FEWHA_ERR_ARG, "noise_sigma must be > 0");
        if (!(geo.gs_height[g] >= 0)) return fail(FEWHA_ERR_ARG, "gs_height must be >= 0");
        w.d = geo.D / w.n;
        w.w = 1.0 / (geo.noise_sigma[g] * geo.noise_sigma[g]);
        w.tx = geo.theta_x[g];
        w.ty = geo.theta_y[g];
        w.H = geo.gs_height[g];
        w.soff = soff;
        w.noff = noff;
        w.moff = moff;
        soff += 2L * w.n * w.n;
        noff += (long)(w.n + 1) * (w.n + 1);
        moff += (long)w.n * w.n;
        // pupil mask: centre of subaperture (i, j) at ((2j+1-n), (2i+1-n)) * d/2;
        // active iff (obstruction*n)^2 <= r^2 <= n^2 in those half-units; a
        // low-order (tip-tilt) sensor, n <= 2, spans the pupil: all active.
        const double inner = (geo.obstruction * w.n) * (geo.obstruction * w.n);
        for (int i = 0; i < w.n; ++i)
            for (int j = 0; j < w.n; ++j) {
                long cy = 2L * i + 1 - w.n, cx = 2L * j + 1 - w.n;
                long r2 = cx * cx + cy * cy;
                o.mask.push_back((w.n <= 2 || (r2 <= (long)w.n * w.n && (double)r2 >= inner)) ? 1 : 0);
            }
        for (long k = w.moff; k < (long)o.mask.size(); ++k) w.nact += o.mask[k];
        // an LGS does not sense tip / tilt: optional filter of its slope means
        w.tt = geo.lgs_tt_filter != 0 && w.H > 0.0 && w.nact > 0;
        o.any_tt = o.any_tt || w.tt;
    }
    o.S = soff;
    o.NW = noff;
    o.NS = moff;

    // mirrors co-located with the layers (L = M, mirror m at layer m's
    // height): the fit samples each layer at its mirror's actuators, and the
    // layer grid also covers the actuator grid
    double thfit = 0.0;
    for (int t = 0; t < o.T; ++t)
        thfit = std::max(thfit, std::max(std::fabs(geo.fit_theta_x[t]), std::fabs(geo.fit_theta_y[t])));
    o.colocated = o.M > 0 && o.M == o.L && !o.moao;   // MOAO mirrors belong to directions
    for (int m = 0; m < o.M && o.colocated; ++m)
        o.colocated = std::fabs(geo.dm_height[m] - prof.height[m]) <= 1e-6 * std::max(1.0, prof.height[m]);

    // layers: extent = union of all footprints (sensors with their cone
    // factor, fitting directions without); spacing E / (n - 1).
    o.lay.resize(o.L);
    long off = 0;
    for (int l = 0; l < o.L; ++l) {
        HostLayer& L = o.lay[l];
        L.n = prof.n_side[l];
        L.J = prof.levels[l];
        L.h = prof.height[l];
        L.cn2 = prof.cn2[l];
        if (!is_pow2(L.n) || L.n < 8 || L.n > 1024) return fail(FEWHA_ERR_ARG, "layer n_side must be a power of two in 8..1024");
        if (L.J < 1 || (L.n >> L.J) < 2) return fail(FEWHA_ERR_ARG, "levels must satisfy 1 <= J and n >> J >= 2");
        if (!(L.cn2 > 0)) return fail(FEWHA_ERR_ARG, "cn2 fractions must be > 0");
        if (!(L.h >= 0)) return fail(FEWHA_ERR_ARG, "layer heights must be >= 0");
        double ext = 0.0;
        for (int g = 0; g < o.G; ++g) {
            const HostWfs& w = o.wfs[g];
            double s = w.H > 0.0 ? 1.0 - L.h / w.H : 1.0;
            if (!(s > 0.0)) return fail(FEWHA_ERR_GEOMETRY, "layer above a laser guide star");
            double th = std::max(std::fabs(w.tx), std::fabs(w.ty));
            ext = std::max(ext, 2.0 * (s * geo.D / 2.0 + th * L.h));
        }
        for (int t = 0; t < o.T; ++t) {
            double th = std::max(std::fabs(geo.fit_theta_x[t]), std::fabs(geo.fit_theta_y[t]));
            ext = std::max(ext, 2.0 * (geo.D / 2.0 + th * L.h));
        }
        if (o.colocated && geo.dm_pitch[l] > 0) {
            const int na = mirror_actuators(geo.D, thfit, geo.dm_height[l], geo.dm_pitch[l]);
            ext = std::max(ext, (na - 1) * geo.dm_pitch[l]);
        }
        L.E = ext;
        L.delta = ext / (L.n - 1);
        L.X0 = -ext / 2.0;
        L.off = off;
        off += (long)L.n * L.n;
    }
    o.N = off;

    // sample and gather tables per (g, l)
    o.tab_off.resize((size_t)o.G * o.L);
    o.gat_off.resize((size_t)o.G * o.L);
    for (int g = 0; g < o.G; ++g)
        for (int l = 0; l < o.L; ++l) {
            const HostWfs& w = o.wfs[g];
            const HostLayer& L = o.lay[l];
            double s = w.H > 0.0 ? 1.0 - L.h / w.H : 1.0;
            o.tab_off[g * o.L + l] = (int)o.cx.size();
            if (!sample_table(geo.D, w.n, s, w.tx, L.h, L.X0, L.delta, L.n, o.cx, o.tx) ||
                !sample_table(geo.D, w.n, s, w.ty, L.h, L.X0, L.delta, L.n, o.cy, o.ty)) {
                snprintf(buf, sizeof buf, "sensor %d footprint leaves the grid of layer %d", g, l);
                return fail(FEWHA_ERR_GEOMETRY, buf);
            }
            int base = o.tab_off[g * o.L + l];
            o.gat_off[g * o.L + l] = (int)o.jlo.size();
            gather_ranges(&o.cx[base], w.n + 1, L.n, o.jlo, o.jhi);
            gather_ranges(&o.cy[base], w.n + 1, L.n, o.ilo, o.ihi);
        }

    // regulariser D (Kolmogorov scaling of the wavelet variance per level)
    // and the level of every coefficient
    o.Dreg.assign(o.N, 0.0);
    o.aD.assign(o.N, 0.0);
    o.level.assign(o.N, 0);
    for (int l = 0; l < o.L; ++l) {
        const HostLayer& L = o.lay[l];
        for (int y = 0; y < L.n; ++y)
            for (int x = 0; x < L.n; ++x) {
                int j = level_of(y, x, L.n, L.J);
                double Dv = reg_diag(o.r0, L.cn2, L.delta, j);
                long i = L.off + (long)y * L.n + x;
                o.Dreg[i] = Dv;
                o.aD[i] = o.alpha * Dv;
                o.level[i] = j;
            }
    }

    // Jacobi diagonal diag(M) = alpha D + sum_g w_g |mask Gamma P_g W^T e_i|^2.
    // Basis functions are tensor products f_y (x) f_x of level-j 1D functions;
    // interpolation is a tensor product too and Gamma^x = (average in y) x
    // (difference in x), Gamma^y the other way round, so the squared norm is
    // sum_{a,b} mask_ab [ (A u)_a^2 (D v)_b^2 + (D u)_a^2 (A v)_b^2 ].
    o.Jdiag = o.aD;
    for (int l = 0; l < o.L; ++l) {
        const HostLayer& L = o.lay[l];
        const int n = L.n;
        for (int j = 1; j <= L.J; ++j) {
            const int m2 = n >> (j - 1);
            std::vector<double> F = level_functions(n, j, o.h, o.g);
            for (int g = 0; g < o.G; ++g) {
                const HostWfs& w = o.wfs[g];
                const int ns = w.n;
                const int base = o.tab_off[g * o.L + l];
                std::vector<double> AU((size_t)m2 * ns), DU((size_t)m2 * ns), AV((size_t)m2 * ns), DV((size_t)m2 * ns);
                std::vector<double> AUl((size_t)m2 * ns), DUl((size_t)m2 * ns), AVl((size_t)m2 * ns), DVl((size_t)m2 * ns);
                std::vector<double> U(ns + 1), V(ns + 1);
                for (int k = 0; k < m2; ++k) {
                    const double* f = &F[(size_t)k * n];
                    for (int i = 0; i <= ns; ++i) {
                        U[i] = f[o.cy[base + i]] * (1.0 - o.ty[base + i]) + f[o.cy[base + i] + 1] * o.ty[base + i];
                        V[i] = f[o.cx[base + i]] * (1.0 - o.tx[base + i]) + f[o.cx[base + i] + 1] * o.tx[base + i];
                    }
                    for (int a = 0; a < ns; ++a) {
                        double au = 0.5 * (U[a] + U[a + 1]), du = U[a + 1] - U[a];
                        double av = 0.5 * (V[a] + V[a + 1]), dv = V[a + 1] - V[a];
                        AU[(size_t)k * ns + a] = au * au;
                        DU[(size_t)k * ns + a] = du * du;
                        AV[(size_t)k * ns + a] = av * av;
                        DV[(size_t)k * ns + a] = dv * dv;
                        AUl[(size_t)k * ns + a] = au;
                        DUl[(size_t)k * ns + a] = du;
                        AVl[(size_t)k * ns + a] = av;
                        DVl[(size_t)k * ns + a] = dv;
                    }
                }
                // T1[a][kx] = sum_b mask[a][b] DV[kx][b],  T2 with AV
                std::vector<double> T1((size_t)ns * m2), T2((size_t)ns * m2);
                const unsigned char* mk = &o.mask[w.moff];
                for (int a = 0; a < ns; ++a)
                    for (int kx = 0; kx < m2; ++kx) {
                        double s1 = 0, s2 = 0;
                        for (int b = 0; b < ns; ++b)
                            if (mk[a * ns + b]) {
                                s1 += DV[(size_t)kx * ns + b];
                                s2 += AV[(size_t)kx * ns + b];
                            }
                        T1[(size_t)a * m2 + kx] = s1;
                        T2[(size_t)a * m2 + kx] = s2;
                    }
                // LGS tip-tilt filter: minus the squared active sums of each
                // slope axis, (sum mask (A u)(D v))^2 + (sum mask (D u)(A v))^2, / n_act
                std::vector<double> T3, T4;
                if (w.tt) {
                    T3.assign((size_t)ns * m2, 0.0);
                    T4.assign((size_t)ns * m2, 0.0);
                    for (int a = 0; a < ns; ++a)
                        for (int kx = 0; kx < m2; ++kx) {
                            double s3 = 0, s4 = 0;
                            for (int b = 0; b < ns; ++b)
                                if (mk[a * ns + b]) {
                                    s3 += DVl[(size_t)kx * ns + b];
                                    s4 += AVl[(size_t)kx * ns + b];
                                }
                            T3[(size_t)a * m2 + kx] = s3;
                            T4[(size_t)a * m2 + kx] = s4;
                        }
                }
                for (int y = 0; y < m2; ++y)
                    for (int x = 0; x < m2; ++x) {
                        if (level_of(y, x, n, L.J) != j) continue;
                        double q = 0;
                        for (int a = 0; a < ns; ++a)
                            q += AU[(size_t)y * ns + a] * T1[(size_t)a * m2 + x] + DU[(size_t)y * ns + a] * T2[(size_t)a * m2 + x];
                        if (w.tt) {
                            double sx = 0, sy = 0;
                            for (int a = 0; a < ns; ++a) {
                                sx += AUl[(size_t)y * ns + a] * T3[(size_t)a * m2 + x];
                                sy += DUl[(size_t)y * ns + a] * T4[(size_t)a * m2 + x];
                            }
                            q -= (sx * sx + sy * sy) / w.nact;
                        }
                        o.Jdiag[L.off + (long)y * n + x] += w.w * q;
                    }
            }
        }
    }

    // modified Jacobi: each coefficient's diagonal times its level's weight
    for (long i = 0; i < o.N; ++i) {
        const int j = o.level[i];
        const double w = (j >= 1 && j <= FEWHA_MAX_JACOBI_LEVELS) ? prof.jacobi_level_weight[j - 1] : 0.0;
        if (w > 0.0) o.Jdiag[i] *= w;
    }

    // ---- mirrors and fitting directions ----
    if (o.M > 0) {
        o.fit_n = geo.fit_n_sub > 0 ? geo.fit_n_sub : o.wfs[0].n;
        double thmax = 0.0;
        for (int t = 0; t < o.T; ++t)
            thmax = std::max(thmax, std::max(std::fabs(geo.fit_theta_x[t]), std::fabs(geo.fit_theta_y[t])));
        o.dm.resize(o.M);
        long aoff = 0;
        for (int m = 0; m < o.M; ++m) {
            HostDm& dm = o.dm[m];
            dm.h = geo.dm_height[m];
            dm.pitch = geo.dm_pitch[m];
            if (!(dm.pitch > 0) || !(dm.h >= 0)) return fail(FEWHA_ERR_ARG, "mirror pitch must be > 0 and height >= 0");
            dm.na = mirror_actuators(geo.D, thmax, dm.h, dm.pitch);
            if (dm.na > 4096) return fail(FEWHA_ERR_ARG, "mirror grid too large");
            dm.A0 = -(dm.na - 1) * dm.pitch / 2.0;
            dm.off = aoff;
            aoff += (long)dm.na * dm.na;
        }
        o.NA = aoff;
        // co-located fit: actuator k of mirror m on layer m's grid (the grids
        // are square and centred, so one table serves both axes)
        if (o.colocated) {
            o.ctab_off.resize(o.M);
            for (int m = 0; m < o.M; ++m) {
                const HostDm& dm = o.dm[m];
                const HostLayer& L = o.lay[m];
                o.ctab_off[m] = (int)o.ccx.size();
                for (int k = 0; k < dm.na; ++k) {
                    int c;
                    double w;
                    if (!bilinear_cell((dm.A0 + k * dm.pitch - L.X0) / L.delta, L.n, c, w))
                        return fail(FEWHA_ERR_GEOMETRY, "a mirror's actuators leave its layer grid");
                    o.ccx.push_back(c);
                    o.ctx.push_back(w);
                }
            }
        }
        o.ftab_off.resize((size_t)o.T * o.L);
        o.dtab_off.resize((size_t)o.T * o.M);
        o.dgat_off.resize((size_t)o.T * o.M);
        for (int t = 0; t < o.T; ++t) {
            double tx = geo.fit_theta_x[t], ty = geo.fit_theta_y[t];
            for (int l = 0; l < o.L; ++l) {
                const HostLayer& L = o.lay[l];
                o.ftab_off[t * o.L + l] = (int)o.fcx.size();
                if (!sample_table(geo.D, o.fit_n, 1.0, tx, L.h, L.X0, L.delta, L.n, o.fcx, o.ftx) ||
                    !sample_table(geo.D, o.fit_n, 1.0, ty, L.h, L.X0, L.delta, L.n, o.fcy, o.fty))
                    return fail(FEWHA_ERR_GEOMETRY, "fitting footprint leaves a layer grid");
            }
            for (int m = 0; m < o.M; ++m) {
                const HostDm& dm = o.dm[m];
                o.dtab_off[t * o.M + m] = (int)o.dcx.size();
                if (!sample_table(geo.D, o.fit_n, 1.0, tx, dm.h, dm.A0, dm.pitch, dm.na, o.dcx, o.dtx) ||
                    !sample_table(geo.D, o.fit_n, 1.0, ty, dm.h, dm.A0, dm.pitch, dm.na, o.dcy, o.dty))
                    return fail(FEWHA_ERR_GEOMETRY, "fitting footprint leaves a mirror grid");
                int base = o.dtab_off[t * o.M + m];
                o.dgat_off[t * o.M + m] = (int)o.djlo.size();
                gather_ranges(&o.dcx[base], o.fit_n + 1, dm.na, o.djlo, o.djhi);
                gather_ranges(&o.dcy[base], o.fit_n + 1, dm.na, o.dilo, o.dihi);
            }
        }
        // closed loop (Alg. 1): the mirrors as every sensor sees them -- shift
        // theta_g h_m and, for a laser guide star, cone factor 1 - h_m/H_g;
        // unavailable (not an error) when a footprint leaves a mirror grid
        o.closed_ok = !o.moao;   // the sensors do not see MOAO mirrors: open loop
        o.wdtab_off.resize((size_t)o.G * o.M);
        for (int g = 0; g < o.G && o.closed_ok; ++g) {
            const HostWfs& w = o.wfs[g];
            for (int m = 0; m < o.M && o.closed_ok; ++m) {
                const HostDm& dm = o.dm[m];
                const double sc = (w.H > 0) ? 1.0 - dm.h / w.H : 1.0;
                o.wdtab_off[g * o.M + m] = (int)o.wdcx.size();
                if (!sample_table(geo.D, w.n, sc, w.tx, dm.h, dm.A0, dm.pitch, dm.na, o.wdcx, o.wdtx) ||
                    !sample_table(geo.D, w.n, sc, w.ty, dm.h, dm.A0, dm.pitch, dm.na, o.wdcy, o.wdty))
                    o.closed_ok = false;
            }
        }
        if (!o.closed_ok) {
            o.wdtab_off.clear();
            o.wdcx.clear();
            o.wdcy.clear();
            o.wdtx.clear();
            o.wdty.clear();
        }
        // eps = 1e-6 * mean diagonal of sum_t P_DM_t^T P_DM_t (MOAO: pairs t = m)
        double dsum = 0.0;
        for (int t = 0; t < o.T; ++t)
            for (int m = 0; m < o.M; ++m) {
                if (o.moao && m != t) continue;
                int base = o.dtab_off[t * o.M + m];
                double sx[2] = {0, 0};
                (void)sx;
                // sum over actuators of sum over nodes of weight^2 = sum over nodes of
                // (sum of squared weights of the 4 corners) = sum_i wy_i^2 * sum_j wx_j^2
                double sy2 = 0, sx2 = 0;
                for (int i = 0; i <= o.fit_n; ++i) {
                    double a = o.dty[base + i], b = o.dtx[base + i];
                    sy2 += (1 - a) * (1 - a) + a * a;
                    sx2 += (1 - b) * (1 - b) + b * b;
                }
                dsum += sy2 * sx2;
            }
        o.fit_eps = 1e-6 * dsum / (double)o.NA;
    }
    return FEWHA_OK;
}

}  // namespace fewha
