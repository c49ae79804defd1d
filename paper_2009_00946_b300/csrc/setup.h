// Host-side geometry of one FEWHA instance (FP64), built once at fewha_create.
#pragma once
#include <string>
#include <vector>

#include "fewha.h"

namespace fewha {

// Layer grid l: n x n nodes X_p = X0 + p*delta (Sec. 2.1 layered model; the
// grid extent covers the union of all sensor and fitting footprints).
struct HostLayer {
    int n = 0, J = 0;
    long off = 0;           // offset in the coefficient vector
    double h = 0, cn2 = 0, E = 0, delta = 0, X0 = 0;
};

// Shack-Hartmann sensor g (Sec. 2.1): n_sub x n_sub subapertures of size d.
struct HostWfs {
    int n = 0;
    long soff = 0;          // slope offset (2 n^2 per sensor)
    long noff = 0;          // node offset ((n+1)^2 per sensor)
    long moff = 0;          // mask / subaperture offset (n^2 per sensor)
    double d = 0, w = 0;    // w = 1 / sigma^2
    int nact = 0;           // active subapertures
    bool tt = false;        // LGS tip-tilt filter on this sensor
    double tx = 0, ty = 0, H = 0;
};

// Deformable mirror m for the fit: na x na actuators A0 + k*pitch.
struct HostDm {
    int na = 0;
    long off = 0;
    double h = 0, pitch = 0, A0 = 0;
};

struct HostSetup {
    int L = 0, G = 0, M = 0, T = 0;          // layers, sensors, mirrors, fitting directions
    bool any_tt = false;                     // some sensor has the LGS tip-tilt filter
    long N = 0, S = 0, NW = 0, NS = 0, NA = 0; // coeffs, slopes, sensor nodes, subapertures, actuators
    int prec = FEWHA_FP32;
    double D = 0, obstruction = 0, r0 = 0, alpha = 0;
    std::vector<HostLayer> lay;
    std::vector<HostWfs> wfs;
    std::vector<HostDm> dm;
    std::vector<unsigned char> mask;         // NS entries

    // bilinear sample tables per (g, l): nodes k = 0..n_g (x uses theta_x, y theta_y)
    std::vector<int> tab_off;                // G*L, offset into cx/cy/tx/ty
    std::vector<int> cx, cy;
    std::vector<double> tx, ty;
    // gather ranges of the transposed interpolation per (g, l): for layer
    // column q the sensor columns j with cx_j in {q-1, q} are [jlo[q], jhi[q]).
    std::vector<int> gat_off;                // G*L, offset into jlo/jhi/ilo/ihi
    std::vector<int> jlo, jhi, ilo, ihi;

    // fitting: pupil nodes (fit_n+1)^2; per (t, l) layer tables and per (t, m)
    // mirror tables (same layout as above), and mirror gather ranges.
    int fit_n = 0;
    double fit_eps = 0;
    std::vector<int> ftab_off, fcx, fcy;     // (T*L): layer sample tables on the pupil grid
    std::vector<double> ftx, fty;
    std::vector<int> dtab_off, dcx, dcy;     // (T*M): mirror sample tables
    std::vector<double> dtx, dty;
    std::vector<int> dgat_off, djlo, djhi, dilo, dihi;   // (T*M): per actuator index
    // closed loop: mirror m sampled at the nodes of sensor g (G*M tables, same
    // layout as the layer tables); closed_ok = every sensor sees inside the mirrors
    // L = M with co-located mirrors: fit = sampling of layer m at mirror m's
    // actuators (per mirror na entries: layer cell and weight along one axis)
    bool colocated = false;
    std::vector<int> ctab_off, ccx;
    std::vector<double> ctx;
    bool closed_ok = false;
    bool moao = false;                       // mirror t is fitted in direction t alone
    std::vector<int> wdtab_off, wdcx, wdcy;
    std::vector<double> wdtx, wdty;

    double h[6], g[6];                       // db3 analysis filters
    std::vector<double> aD;                  // alpha * D, N entries
    std::vector<double> Jdiag;               // diag(M), N entries
    std::vector<double> Dreg;                // D (without alpha), N entries
    std::vector<int> level;                  // DWT level of every coefficient, N entries
};

// Validate the inputs, build every table and the Jacobi diagonal.  Returns a
// FEWHA status; on failure err holds the message.
int build_setup(const fewha_geometry& geo, const fewha_profile& prof, HostSetup& out, std::string& err);

// Diagonal of the regulariser D for a coefficient of wavelet level j on a
// layer with Cn^2 fraction cn2 and grid spacing delta (Sec. 2.2: the
// Kolmogorov scaling r0^{5/3} / (cn2 delta^{5/3} 2^{11 j / 3})).
double reg_diag(double r0, double cn2, double delta, int j);

// db3 taps from the closed form in radicals.
void db3_taps(double h[6], double g[6]);

}  // namespace fewha
