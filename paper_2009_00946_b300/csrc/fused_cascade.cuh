// Layer phase of the fused frame kernel in its level-stacked form: the 2D
// periodic db3 DWT of a layer (Sec. 2.2, Mallat layout: each level transforms
// rows then columns of the LL block) distributed over a thread-block cluster
// with ONE exchange through distributed shared memory per transform instead
// of one cluster barrier per level.
//
// Each level of the 2D transform is separable, L_j X L_j^T with L_j the 1D
// analysis of length m_j = n / 2^{j-1}.  Write Lo_j = H_j ... H_1 and
// Hi_j = G_j Lo_{j-1} for the 1D lowpass chain and the level-j highpass.  Then
// the level-j bands of W X are Lo_j X Hi_j^T (top right), Hi_j X Lo_j^T (bottom
// left), Hi_j X Hi_j^T (bottom right) and, at j = J, Lo_J X Lo_J^T.  So:
//   1. every column of X goes through the 1D cascade keeping ALL levels:
//      U = [Lo_1; Hi_1; Lo_2; Hi_2; ...; Lo_J; Hi_J] X   (T_U = 2n(1 - 2^-J) rows),
//      local to the CTA that holds those columns (column stripes of R = n / C);
//   2. the rows of U are dealt to the CTAs (host-balanced ownership tables);
//      every value of U is stored straight into its owner's shared memory as
//      the column cascade produces it, and one cluster barrier completes the
//      exchange (no gather step);
//   3. row u of kind Lo_j (j < J) needs Hi_j applied (one Mallat row segment),
//      rows of kind Hi_j or Lo_J need Lo_j and Hi_j (one segment of 2 n / 2^j):
//      a 1D lowpass cascade of depth j - 1, then one analysis step.
// The CTA then owns a set of Mallat row segments; the Alg. 2 update is
// elementwise on them.  The inverse W^T = W^{-1} runs the transposes in
// reverse order: row synthesis of every owned row (back to the rows of U, the
// finest level stored straight into the column stripes' owners), one cluster
// barrier, and the column synthesis
//   X = sum_j Lo_{j-1}^T (H_j^T U_{Lo_j} + G_j^T U_{Hi_j})   (Horner, coarse to fine).
//
// Shared memory of a layer item (float offsets from sm, set by the plan):
//   v_z  Z     the column stripe, n rows x R, row-major (R contiguous)
//   v_t  T     row-cascade intermediates, S x n/2; column-synthesis ping-pong
//   v_u  Ucol  the stripe's columns of every row of U, T_U x R, written by the
//              rows' owners in the inverse exchange; before that (in program
//              order, and before the first cluster barrier the other CTAs
//              wait on) it holds the staged sensor fields and then the column
//              cascade's lowpass levels a_1 .. a_{J-1}
//   v_r  Urow  the CTA's rows of U, S x n, written by every CTA in the forward
//              exchange; then the row cascades' workspace
//   v_c  Zc    the CTA's coefficients: its Mallat row segments in slot order
//   ltab       gather tables xt [G][R][KG], yt [G][n][KG] (int2), then at
//   v_tab      the cascade tables (ints): header [20] = S, ncoef, T_U, J,
//              cnt[16] (slots of depth >= level i at cnt[i-1]); slot entries
//              int4 (u, j | isA << 8, Mallat offset in the layer, Zc offset),
//              sorted by depth descending; own map [T_U] (owner << 16 | slot);
//              the Mallat offset in the layer of every owned coefficient.

// Staging boxes, gather tables and cascade tables of the cached layer item
// for this rank (asynchronous copies; the caller waits and synchronises).
__device__ void layer_tables_v1(const FParams& P, int rank, const CtaCache* cc, float* sm) {
    const int tid = threadIdx.x, NT = blockDim.x;
    const LItem& LI = cc->LI;
    const FInst& I = cc->IL;
    const int n = cc->n, R = n / P.C, c0 = rank * R, G = I.G, L = I.L, l = LI.l, KG = I.KG;
    int* sgi = sgi_buf();
    if (tid < G) {
        // sensor tid: rows [x, y), columns [z, w) of its node grid; each row is
        // copied from the 16-byte boundary at or below its first column, so a
        // row slot of W floats holds the box row at offset (s0 + i np1) & 3
        auto width = [](int4 b) { return (b.y > b.x && b.w > b.z) ? ((b.w - b.z + 6) & ~3) : 0; };
        int so = 0;
        for (int g = 0; g < tid; ++g) {
            const int4 b = P.stg4[LI.stg + rank * G + g];
            so += (b.y - b.x) * width(b);
        }
        const int4 b = P.stg4[LI.stg + rank * G + tid];
        const int W = width(b);
        sgi[tid * 8 + 0] = b.x;
        sgi[tid * 8 + 1] = W ? b.y : b.x;
        sgi[tid * 8 + 2] = so;
        sgi[tid * 8 + 3] = I.wfs_n[tid] + 1;
        sgi[tid * 8 + 4] = b.z;
        sgi[tid * 8 + 5] = W;
        sgi[tid * 8 + 6] = I.wfs_noff[tid] + b.z;
        // row of a staging piece by multiply-high with ceil(2^32 / (W / 4)),
        // exact for the small piece counts here; W / 4 = 1 is marked 0
        const unsigned w4 = (unsigned)W >> 2;
        sgi[tid * 8 + 7] = w4 > 1 ? (int)(unsigned)(((1ull << 32) + w4 - 1) / w4) : 0;
    }
    int2* xt = (int2*)(sm + P.ltab_off);          // [g][c][KG]  (j, w), own columns
    int2* yt = xt + P.G_max * P.v_rmax * KG;      // [g][p][KG]  (i, w), every row
    for (int e = tid; e < G * R * KG; e += NT) {
        const int g = e / (R * KG), r = e - g * R * KG;
        cp_async8(xt + e, I.gtab + I.gtab_off[g * L + l] + c0 * KG + r);
    }
    for (int e = tid; e < G * n * KG; e += NT) {
        const int g = e / (n * KG), r = e - g * n * KG;
        cp_async8(yt + e, I.gtab + I.gtab_off[g * L + l] + n * KG + r);
    }
    // cascade tables: this rank's header and slots, then the own map
    const int* blk = P.cshape + LI.csh;
    const int* rb = blk + blk[4 + rank];
    const int* om = blk + blk[4 + P.C];
    int* tab = (int*)(sm + P.v_tab);
    const int S = __ldg(rb), hs = 20 + 4 * S;   // header + slots (ints)
    for (int e = tid; e < hs; e += NT) cp_async4(tab + e, rb + e);
    const int TU = __ldg(blk), nc = __ldg(rb + 1);
    int* own = tab + 20 + 4 * P.v_smax;
    for (int e = tid; e < TU; e += NT) cp_async4(own + e, om + e);
    int* gix = own + P.v_tumax;
    for (int e = tid; e < nc; e += NT) cp_async4(gix + e, rb + hs + e);
}

// The gather tables of a freshly staged layer item, rewritten once for the
// gather below: a row entry's sensor row i becomes the offset in the staged
// fields of that row's column 0 (its slot + (i - ilo) W + the row's 16-byte
// shift - jlo), clamped to a staged row, and a padding column entry (weight
// 0) points at a staged column, so that the gather does no index arithmetic
// per tap.  The caller synchronises the CTA before the tables are read.
__device__ __forceinline__ void pt_tables_to_offsets(const int* sgi, int2* xt, int2* yt, int G, int n, int R, int KG) {
    const int tid = threadIdx.x, NT = blockDim.x;
    for (int e = tid; e < G * n * KG; e += NT) {
        const int g = e / (n * KG);
        const int ilo = sgi[g * 8], ihi = sgi[g * 8 + 1];
        if (ihi <= ilo) continue;
        const int np1 = sgi[g * 8 + 3], jlo = sgi[g * 8 + 4], W = sgi[g * 8 + 5], s0 = sgi[g * 8 + 6];
        int2 ye = yt[e];
        const int i = min(max(ye.x, ilo), ihi - 1);
        ye.x = sgi[g * 8 + 2] + (i - ilo) * W + ((s0 + i * np1) & 3) - jlo;
        yt[e] = ye;
    }
    for (int e = tid; e < G * R * KG; e += NT) {
        const int g = e / (R * KG);
        const int2 xe = xt[e];
        if (__int_as_float(xe.y) == 0.f) xt[e] = make_int2(sgi[g * 8 + 4], xe.y);
    }
}

// KGT (j, w) or (offset, w) entries at e: two per 16-byte load when KGT is even
template <int KGT>
__device__ __forceinline__ void pt_entries(const int2* e, int* idx, float* w) {
    if constexpr (KGT % 2 == 0) {
#pragma unroll
        for (int b = 0; b < KGT; b += 2) {
            const int4 v = *reinterpret_cast<const int4*>(e + b);
            idx[b] = v.x;
            w[b] = __int_as_float(v.y);
            idx[b + 1] = v.z;
            w[b + 1] = __int_as_float(v.w);
        }
    } else {
#pragma unroll
        for (int b = 0; b < KGT; ++b) {
            const int2 v = e[b];
            idx[b] = v.x;
            w[b] = __int_as_float(v.y);
        }
    }
}

// P^T gather into the column stripe from the rewritten tables: thread
// (column c, rows rr0, rr0 + rstep, ...); per sensor the column entries are
// read once for all its rows.
template <int KGT>
__device__ __forceinline__ void pt_gather_cols(const int* sgi, const float* stg, const int2* xt, const int2* yt,
                                               float* Z, int G, int n, int R) {
    constexpr int kRows = 8;
    const int tid = threadIdx.x, NT = blockDim.x;
    const int rstep = NT / R;          // R <= NT (a power of two)
    const int q = tid % R, rr0 = tid / R;
    if (rr0 >= rstep) return;
    for (int rb = rr0; rb < n; rb += rstep * kRows) {
        float acc[kRows];
#pragma unroll
        for (int u = 0; u < kRows; ++u) acc[u] = 0.f;
        for (int g = 0; g < G; ++g) {
            if (sgi[g * 8 + 1] <= sgi[g * 8]) continue;
            int xj[KGT];
            float xw[KGT];
            pt_entries<KGT>(xt + (g * R + q) * KGT, xj, xw);
#pragma unroll
            for (int u = 0; u < kRows; ++u) {
                const int rr = rb + u * rstep;
                if (rr >= n) break;
                int yo[KGT];
                float yw[KGT];
                pt_entries<KGT>(yt + (g * n + rr) * KGT, yo, yw);
#pragma unroll
                for (int a = 0; a < KGT; ++a) {
                    const float* row = stg + yo[a];
                    float racc = 0.f;
#pragma unroll
                    for (int b = 0; b < KGT; ++b)
                        if (FEWHA_IN_SMEM(row + xj[b], 4, kDbgPtRead)) racc += xw[b] * row[xj[b]];
                    acc[u] += yw[a] * racc;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
            const int rr = rb + u * rstep;
            if (rr < n) Z[rr * R + q] = acc[u];
        }
    }
}

// Row offset of level j's a block in U (its d block follows, half_j rows on).
__device__ __forceinline__ int casc_base(int n, int j) { return 2 * n - 2 * (n >> (j - 1)); }

// 1. column cascade of the stripe, every level kept.  Level j's lowpass
// output a_j (j < J) stays here (A, the next level's input); every value of
// U goes straight to the owner of its row: row u's slot in CTA own[u] >> 16,
// columns c0 .. c0 + R - 1 of that slot (rUrow: the CTAs' Urow).
__device__ __forceinline__ void casc_cols_fwd(const FParams& P, const float* Z, float* A, float* const* rUrow,
                                              const int* own, int n, int J, int R, int lR, int c0) {
    const int tid = threadIdx.x, NT = blockDim.x;
    for (int j = 1; j <= J; ++j) {
        const int m = n >> (j - 1), half = m >> 1, mask = m - 1;
        const float* in = (j == 1) ? Z : A + (n - (n >> (j - 2))) * R;
        float* oa = A + (n - (n >> (j - 1))) * R;
        const int ub = casc_base(n, j);
        if (lR >= 2) {
            // four neighbouring columns per thread: 16-byte loads and stores
            const int l4 = lR - 2, items = half << l4;
            for (int e = tid; e < items; e += NT) {
                const int k = e >> l4, c = (e & ((1 << l4) - 1)) << 2;
                float4 a = make_float4(0.f, 0.f, 0.f, 0.f), d = a;
#pragma unroll
                for (int t = 0; t < 6; ++t) {
                    const float4 v = *reinterpret_cast<const float4*>(in + ((2 * k + t) & mask) * R + c);
                    a.x += P.h[t] * v.x;
                    a.y += P.h[t] * v.y;
                    a.z += P.h[t] * v.z;
                    a.w += P.h[t] * v.w;
                    d.x += P.g[t] * v.x;
                    d.y += P.g[t] * v.y;
                    d.z += P.g[t] * v.z;
                    d.w += P.g[t] * v.w;
                }
                if (j < J) *reinterpret_cast<float4*>(oa + k * R + c) = a;
                const int wa = own[ub + k], wd = own[ub + half + k];
                if (FEWHA_IN(wa >> 16, P.C, 1, kDbgCascOwn) && FEWHA_IN((wa & 0xffff) * n + c0 + c, P.v_c - P.v_r, 4, kDbgCascOwn))
                    *reinterpret_cast<float4*>(rUrow[wa >> 16] + (wa & 0xffff) * n + c0 + c) = a;
                if (FEWHA_IN(wd >> 16, P.C, 1, kDbgCascOwn) && FEWHA_IN((wd & 0xffff) * n + c0 + c, P.v_c - P.v_r, 4, kDbgCascOwn))
                    *reinterpret_cast<float4*>(rUrow[wd >> 16] + (wd & 0xffff) * n + c0 + c) = d;
            }
        } else {
            const int items = half << lR;
            for (int e = tid; e < items; e += NT) {
                const int k = e >> lR, c = e & (R - 1);
                float a = 0.f, d = 0.f;
#pragma unroll
                for (int t = 0; t < 6; ++t) {
                    const float v = in[((2 * k + t) & mask) * R + c];
                    a += P.h[t] * v;
                    d += P.g[t] * v;
                }
                if (j < J) oa[e] = a;
                const int wa = own[ub + k], wd = own[ub + half + k];
                if (FEWHA_IN(wa >> 16, P.C, 1, kDbgCascOwn) && FEWHA_IN((wa & 0xffff) * n + c0 + c, P.v_c - P.v_r, 1, kDbgCascOwn))
                    rUrow[wa >> 16][(wa & 0xffff) * n + c0 + c] = a;
                if (FEWHA_IN(wd >> 16, P.C, 1, kDbgCascOwn) && FEWHA_IN((wd & 0xffff) * n + c0 + c, P.v_c - P.v_r, 1, kDbgCascOwn))
                    rUrow[wd >> 16][(wd & 0xffff) * n + c0 + c] = d;
            }
        }
        __syncthreads();
    }
}

// Copy `rows` rows of R = 2^lR floats: dst(r)[x] <- src(r)[x] (16-byte pieces
// when R >= 4 and vec; the source may be another CTA's shared memory).  Each
// thread issues the loads of two pieces before their stores.
template <typename SrcFn, typename DstFn>
__device__ __forceinline__ void casc_copy(int rows, int lR, bool vec, SrcFn src, DstFn dst) {
    const int tid = threadIdx.x, NT = blockDim.x;
    if (vec && lR >= 2) {
        const int l4 = lR - 2, m4 = (1 << l4) - 1, items = rows << l4;
        for (int e0 = tid; e0 < items; e0 += 2 * NT) {
            const int e1 = e0 + NT;
            const float4 a = *reinterpret_cast<const float4*>(src(e0 >> l4) + 4 * (e0 & m4));
            float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e1 < items) b = *reinterpret_cast<const float4*>(src(e1 >> l4) + 4 * (e1 & m4));
            *reinterpret_cast<float4*>(dst(e0 >> l4) + 4 * (e0 & m4)) = a;
            if (e1 < items) *reinterpret_cast<float4*>(dst(e1 >> l4) + 4 * (e1 & m4)) = b;
        }
    } else {
        const int m = (1 << lR) - 1, items = rows << lR;
        for (int e = tid; e < items; e += NT) dst(e >> lR)[e & m] = src(e >> lR)[e & m];
    }
}

// 3. row cascades of the owned rows (Urow, stride n): coefficients into Zc.
// Level i reads Urow (i odd) or T (stride n/2) and writes the other one.
__device__ __forceinline__ void casc_rows_fwd(const FParams& P, const int* tab, float* Urow, float* T, float* Zc, int n) {
    const int tid = threadIdx.x, NT = blockDim.x;
    const int4* slots = reinterpret_cast<const int4*>(tab + 20);
    const int depth = tab[0] > 0 ? (slots[0].y & 255) : 0;
    for (int i = 1; i <= depth; ++i) {
        // outputs k0, k0 + 1 (k0 even) per thread from inputs 2 k0 .. 2 k0 + 7
        // (two 16-byte loads; half >= 2 at every level a row reaches)
        const int m = n >> (i - 1), half = m >> 1, mask = m - 1, lh = 31 - __clz(half);
        const float* in = (i & 1) ? Urow : T;
        const int ins = (i & 1) ? n : (n >> 1);
        float* out = (i & 1) ? T : Urow;
        const int outs = (i & 1) ? (n >> 1) : n;
        const int items = tab[4 + i - 1] << (lh - 1);
        for (int e = tid; e < items; e += NT) {
            const int s = e >> (lh - 1), k0 = (e & ((half >> 1) - 1)) << 1;
            const int4 sl = slots[s];
            const float* x = in + s * ins;
            const float4 q0 = *reinterpret_cast<const float4*>(x + 2 * k0);
            const float4 q1 = *reinterpret_cast<const float4*>(x + ((2 * k0 + 4) & mask));
            const float v[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
            float lo0 = 0.f, lo1 = 0.f;
#pragma unroll
            for (int t = 0; t < 6; ++t) {
                lo0 += P.h[t] * v[t];
                lo1 += P.h[t] * v[t + 2];
            }
            const int j = sl.y & 255;
            if (j > i) {
                *reinterpret_cast<float2*>(out + s * outs + k0) = make_float2(lo0, lo1);
            } else {
                float hi0 = 0.f, hi1 = 0.f;
#pragma unroll
                for (int t = 0; t < 6; ++t) {
                    hi0 += P.g[t] * v[t];
                    hi1 += P.g[t] * v[t + 2];
                }
                if (sl.y >> 8) {
                    *reinterpret_cast<float2*>(Zc + sl.w + k0) = make_float2(hi0, hi1);
                } else {
                    *reinterpret_cast<float2*>(Zc + sl.w + k0) = make_float2(lo0, lo1);
                    *reinterpret_cast<float2*>(Zc + sl.w + half + k0) = make_float2(hi0, hi1);
                }
            }
        }
        __syncthreads();
    }
}

// Inverse 1. row synthesis of the owned rows from their coefficients (Zc),
// coarse to fine; level 1's outputs (the rows of U) go straight to the
// column stripes' owners: entry x of row u to CTA x >> lR, Ucol row u, column
// x & (R - 1) (rUcol: the CTAs' Ucol).
__device__ __forceinline__ void casc_rows_inv(const FParams& P, const int* tab, const float* Zc, float* Urow, float* T,
                                              float* const* rUcol, int n, int R, int lR) {
    const int tid = threadIdx.x, NT = blockDim.x;
    const int4* slots = reinterpret_cast<const int4*>(tab + 20);
    const int depth = tab[0] > 0 ? (slots[0].y & 255) : 0;
    for (int i = depth; i >= 1; --i) {
        // outputs 2 k0 .. 2 k0 + 3 (k0 even) per thread from the a and d
        // entries k0 - 2 .. k0 + 1 (periodic)
        const int half = n >> i, hmask = half - 1, lh = 31 - __clz(half);
        const float* prev = ((i + 1) & 1) ? Urow : T;   // level i + 1's output
        const int ps = ((i + 1) & 1) ? n : (n >> 1);
        float* out = (i & 1) ? Urow : T;
        const int outs = (i & 1) ? n : (n >> 1);
        const int items = tab[4 + i - 1] << (lh - 1);
        for (int e = tid; e < items; e += NT) {
            const int s = e >> (lh - 1), k0 = (e & ((half >> 1) - 1)) << 1;
            const int4 sl = slots[s];
            const int j = sl.y & 255;
            const bool isA = (sl.y >> 8) != 0;
            float a[4], d[4];   // entries k0 - 2 + t
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int k = (k0 - 2 + t) & hmask;
                if (j == i) {
                    a[t] = isA ? 0.f : Zc[sl.w + k];
                    d[t] = Zc[sl.w + (isA ? 0 : half) + k];
                } else {
                    a[t] = prev[s * ps + k];
                    d[t] = 0.f;
                }
            }
            float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int sg = 0; sg < 3; ++sg) {
                // output pair k0 takes entry k0 - sg (index 2 - sg), pair k0 + 1 entry k0 + 1 - sg
                o.x += P.h[2 * sg] * a[2 - sg] + P.g[2 * sg] * d[2 - sg];
                o.y += P.h[2 * sg + 1] * a[2 - sg] + P.g[2 * sg + 1] * d[2 - sg];
                o.z += P.h[2 * sg] * a[3 - sg] + P.g[2 * sg] * d[3 - sg];
                o.w += P.h[2 * sg + 1] * a[3 - sg] + P.g[2 * sg + 1] * d[3 - sg];
            }
            const int x = 2 * k0;
            if (i > 1) {
                *reinterpret_cast<float4*>(out + s * outs + x) = o;
            } else if (lR >= 2) {
                if (FEWHA_IN(x >> lR, P.C, 1, kDbgCascCol) && FEWHA_IN(sl.x * R + (x & (R - 1)), P.v_r - P.v_u, 4, kDbgCascCol))
                    *reinterpret_cast<float4*>(rUcol[x >> lR] + sl.x * R + (x & (R - 1))) = o;
            } else {
                const float ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (FEWHA_IN((x + t) >> lR, P.C, 1, kDbgCascCol) &&
                        FEWHA_IN(sl.x * R + ((x + t) & (R - 1)), P.v_r - P.v_u, 1, kDbgCascCol))
                        rUcol[(x + t) >> lR][sl.x * R + ((x + t) & (R - 1))] = ov[t];
            }
        }
        __syncthreads();
    }
}

// Inverse 3. column synthesis of the stripe from the gathered U columns,
// coarse to fine (level j writes Z when j is odd, else T, both [row][R]);
// returns the buffer holding X (= Z).
__device__ __forceinline__ void casc_cols_inv(const FParams& P, const float* U, float* Z, float* T, int n, int J, int R, int lR) {
    const int tid = threadIdx.x, NT = blockDim.x;
    for (int j = J; j >= 1; --j) {
        const int half = n >> j, hmask = half - 1;
        const float* ua = U + casc_base(n, j) * R;
        const float* ud = ua + half * R;
        const float* prev = ((j + 1) & 1) ? Z : T;
        float* out = (j & 1) ? Z : T;
        const bool add = j < J;
        const int items = half << lR;
        for (int e = tid; e < items; e += NT) {
            const int kk = e >> lR, c = e & (R - 1);
            float ox = 0.f, oy = 0.f;
#pragma unroll
            for (int sg = 0; sg < 3; ++sg) {
                const int k = (kk - sg) & hmask;
                const float a = ua[k * R + c] + (add ? prev[k * R + c] : 0.f);
                const float d = ud[k * R + c];
                ox += P.h[2 * sg] * a + P.g[2 * sg] * d;
                oy += P.h[2 * sg + 1] * a + P.g[2 * sg + 1] * d;
            }
            out[(2 * kk) * R + c] = ox;
            out[(2 * kk + 1) * R + c] = oy;
        }
        __syncthreads();
    }
}


// The layer phase in its level-stacked form (same modes and outputs as
// layer_phase).  No CTA reads another's shared memory, and every store into
// another CTA's shared memory precedes a cluster barrier that CTA waits on,
// so the phase needs no barrier at its end.
__device__ void layer_phase_v1(const FParams& P, int li, int mode, int k, float* sm, float* const (*rem)[kMaxC],
                               cg::cluster_group& cl, double* red, double* sh, CtaCache* cc, bool end_sync) {
    const int tid = threadIdx.x, NT = blockDim.x;
    fmark(P, 10);
    const bool fresh = cc->lkey != li;
    if (P.shared_tables && tid == 0) cc->wtab = 0;
    if (fresh) {
        __syncthreads();
        if (tid == 0) layer_desc(P, li, cc);
        __syncthreads();
    }
    const bool tabs = cc->ltkey != li;
    const FInst& I = cc->IL;
    const int C = P.C, rank = (int)cl.block_rank();
    const int n = cc->n, J = cc->J, off = cc->off;
    const int R = n / C, c0 = rank * R, lR = 31 - __clz(R);
    const int G = I.G, KG = I.KG;
    const int* sgi = sgi_buf();
    float* Z = sm + P.v_z;
    float* T = sm + P.v_t;
    float* Ucol = sm + P.v_u;
    float* Urow = sm + P.v_r;
    float* Zc = sm + P.v_c;
    float* stg = Ucol;
    const int* tab = (const int*)(sm + P.v_tab);
    const int2* xt = (const int2*)(sm + P.ltab_off);
    const int2* yt = xt + P.G_max * P.v_rmax * KG;

    // ---- P^T: gather of the sensor fields into the own columns ----
    {
        if (tabs) {
            layer_tables_v1(P, rank, cc, sm);
            __syncthreads();   // the staging boxes
        }
        for (int g = 0; g < G; ++g) {
            const int ilo = sgi[g * 8], rows = sgi[g * 8 + 1] - ilo, W = sgi[g * 8 + 5];
            if (rows <= 0 || W == 0) continue;
            const int np1 = sgi[g * 8 + 3], s0 = sgi[g * 8 + 6], w4 = W >> 2;
            const unsigned mg = (unsigned)sgi[g * 8 + 7];
            float* dst = stg + sgi[g * 8 + 2];
            for (int e = tid; e < rows * w4; e += NT) {
                const int rr = mg ? (int)__umulhi((unsigned)e, mg) : e, x = e - rr * w4;
                const int a0 = (s0 + (ilo + rr) * np1) & ~3;
                // (the field buffer carries 8 floats past NW for the 16-byte rows)
                if (FEWHA_IN(a0 + 4 * x, I.NW + 8, 4, kDbgStgSrc)) cp_async16(dst + rr * W + 4 * x, I.psi + a0 + 4 * x);
            }
        }
        if (mode == kLpIter && tid < 32 && I.preA_cta < 0) {
            ScalA A;
            if (cc->pre_k == k) {
                A.rho = cc->pre[0];
                A.beta = cc->pre[1];
                A.t = cc->pre[2];
                A.aold = cc->pre[3];
                A.mh = (float)cc->pre[4];
                A.ml = (float)cc->pre[5];
            } else {
                alg2_part_a(P, I, k, A);
            }
            alg2_part_b(P, I, k, A, sh);
        }
        cp_async_wait_all();
        if (tabs && tid == 0) cc->ltkey = li;
        __syncthreads();
        if (cc->ltx != li) {   // tables copied here or at launch start: rewritten once
            pt_tables_to_offsets(sgi, const_cast<int2*>(xt), const_cast<int2*>(yt), G, n, R, KG);
            __syncthreads();
            if (tid == 0) cc->ltx = li;
        }

        if (I.tt_any) {
            // LGS tip-tilt filter (R15): Gamma^T C^{-1} s = Gamma^T (w mask s) -
            // (w / n_act) (M_x Gamma^T (mask 1_x) + M_y Gamma^T (mask 1_y)) with
            // M the sensor's masked slope sums (from its tiles' partials): the
            // staged fields of a filtered sensor get the rank-2 term here
            float* ttc = reinterpret_cast<float*>(red);   // [g][2]
            const int wid = tid >> 5, lane = tid & 31;
            if (wid < G) {
                float cx = 0.f, cy = 0.f;
                if (I.tt[wid]) {
                    const int2 tr = I.tt_tiles[wid];
                    float xh = 0.f, xl = 0.f, yh = 0.f, yl = 0.f;
                    for (int e = lane; e < tr.y; e += 32) {
                        const float4 v = __ldcg(P.tpart + tr.x + e);
                        df_add(xh, xl, v.x, v.y);
                        df_add(yh, yl, v.z, v.w);
                    }
                    warp_df_sum(xh, xl);
                    warp_df_sum(yh, yl);
                    const double f = (double)I.wfs_w[wid] / (double)I.nact[wid];
                    cx = (float)(f * df_to_double(xh, xl));
                    cy = (float)(f * df_to_double(yh, yl));
                }
                if (lane == 0) {
                    ttc[2 * wid] = cx;
                    ttc[2 * wid + 1] = cy;
                }
            }
            __syncthreads();
            for (int g = 0; g < G; ++g) {
                if (!I.tt[g]) continue;
                const int ilo = sgi[g * 8], ihi = sgi[g * 8 + 1], W = sgi[g * 8 + 5];
                if (ihi <= ilo || W == 0) continue;
                const int np1 = sgi[g * 8 + 3], jlo = sgi[g * 8 + 4], s0 = sgi[g * 8 + 6];
                const int jhi = P.stg4[cc->LI.stg + rank * G + g].w;   // staged columns [jlo, jhi)
                const float cx = ttc[2 * g], cy = ttc[2 * g + 1];
                float* dst = stg + sgi[g * 8 + 2];
                // only nodes next to a mask edge have a nonzero term: the sensor's
                // list of them (node, Gamma^T (mask 1_x), Gamma^T (mask 1_y))
                const int2 nr = I.tt_nzr[g];
                for (int e = tid; e < nr.y; e += NT) {
                    const int4 nz = __ldg(I.tt_nz + nr.x + e);
                    const int i = nz.x / np1, j = nz.x - i * np1;
                    if (i < ilo || i >= ihi || j < jlo || j >= jhi) continue;
                    if (!FEWHA_IN_SMEM(dst + (i - ilo) * W + ((s0 + i * np1) & 3) + (j - jlo), 4, kDbgTT)) continue;
                    dst[(i - ilo) * W + ((s0 + i * np1) & 3) + (j - jlo)] -=
                        cx * __int_as_float(nz.y) + cy * __int_as_float(nz.z);
                }
            }
            __syncthreads();
        }
        fmark(P, 11);
        switch (KG) {
            case 1: pt_gather_cols<1>(sgi, stg, xt, yt, Z, G, n, R); break;
            case 2: pt_gather_cols<2>(sgi, stg, xt, yt, Z, G, n, R); break;
            case 3: pt_gather_cols<3>(sgi, stg, xt, yt, Z, G, n, R); break;
            default: pt_gather_cols<4>(sgi, stg, xt, yt, Z, G, n, R); break;
        }
    }

    // ---- forward W: column cascade, exchange, row cascades ----
    const bool pub = (mode == kLpIter) && I.preA_cta >= 0;
    unsigned long long wa = 0ull, wa2 = 0ull, wb = 0ull, wb2 = 0ull;
    if (pub && tid == 0) {
        ld_relaxed_v2(I.pubAB + (k & 1) * 4, wa, wa2);
        ld_relaxed_v2(I.pubAB + (k & 1) * 4 + 2, wb, wb2);
    }
    fmark(P, 12);
    __syncthreads();   // the stripe (and the staged fields are no longer read: Ucol may be written)
    casc_cols_fwd(P, Z, Ucol, rem[0], tab + 20 + 4 * P.v_smax, n, J, R, lR, c0);
    fmark(P, 50);
    cl.sync();         // 2. every CTA's stores into this CTA's rows of U have landed
    fmark(P, 51);
    casc_rows_fwd(P, tab, Urow, T, Zc, n);
    fmark(P, 13);

    // ---- elementwise (Alg. 1 restart / Alg. 2 update) on the owned coefficients ----
    const bool last = (mode == kLpIter) && (k + 1 >= P.n_iter);
    const bool make_z = (mode == kLpRhsStart) || (mode == kLpReplStart) || (mode == kLpIter && !last);
    Acc2 rho_p, dz_p;
    const int ncoef = tab[1];
    const int* gix = tab + 20 + 4 * P.v_smax + P.v_tumax;
    float* st = (P.v_st >= 0) ? sm + P.v_st : nullptr;   // resident r, p, q, c, J^{-1}, alpha D
    const int sts = P.v_sts;
    if (mode == kLpIter) {
        constexpr int kE = 4;
        float vr[kE], vp[kE], vq[kE], vc[kE], vj[kE], va[kE];
        int gi[kE];
        auto load = [&](int e0) {
#pragma unroll
            for (int u = 0; u < kE; ++u) {
                const int e = e0 + u * NT;
                if (e < ncoef && FEWHA_IN(off + gix[e], I.N, 1, kDbgCoef)) {
                    const int i = off + gix[e];
                    gi[u] = i;
                    if (st) {
                        vr[u] = st[e];
                        vp[u] = st[sts + e];
                        vq[u] = st[2 * sts + e];
                        vc[u] = st[3 * sts + e];
                        vj[u] = st[4 * sts + e];
                        va[u] = st[5 * sts + e];
                    } else {
                        vr[u] = I.r[i];
                        vp[u] = I.p[i];
                        vq[u] = I.q[i];
                        vc[u] = I.c[i];
                        vj[u] = __ldg(I.Jinv + i);
                        va[u] = __ldg(I.aD + i);
                    }
                }
            }
        };
        load(tid);
        if (pub) {
            if (tid == 0) {
                const unsigned want = (unsigned)k + 1u;
                const long long t0 = clock64();
                bool ok = true;
                while ((unsigned)(wa >> 32) != want || (unsigned)(wa2 >> 32) != want ||
                       (unsigned)(wb >> 32) != want || (unsigned)(wb2 >> 32) != want) {
                    if (clock64() - t0 > P.budget) {
                        ok = false;
                        break;
                    }
                    __nanosleep(32);
                    ld_relaxed_v2(I.pubAB + (k & 1) * 4, wa, wa2);
                    ld_relaxed_v2(I.pubAB + (k & 1) * 4 + 2, wb, wb2);
                }
                sh[0] = ok ? __hiloint2double((int)(unsigned)wa, (int)(unsigned)wa2) : 0.0;
                sh[1] = ok ? __hiloint2double((int)(unsigned)wb, (int)(unsigned)wb2) : 0.0;
                if (!ok) atomicOr(P.errw, kErrTimeout);
            }
            __syncthreads();
        }
        fmark(P, 17);
        const double alpha = sh[0], beta = sh[1];
        if (!pub && tid == 0 && li == I.l0 && rank == 0) {
            double* swp = I.scal + (k & 1) * 2;
            swp[0] = sh[2];
            swp[1] = sh[5];
            if (sh[4] != 0.0) atomicOr(P.errw, kErrBreakdown);
            if (I.sc_out) {
                I.sc_out[kRho] = sh[2];
                I.sc_out[kMu] = sh[3];
                I.sc_out[kBeta] = beta;
                I.sc_out[kAlphaK] = alpha;
            }
        }
        const float fa = (float)alpha, fb = (float)beta;
        for (int e0 = tid; e0 < ncoef; e0 += kE * NT) {
            if (e0 != tid) load(e0);
#pragma unroll
            for (int u = 0; u < kE; ++u) {
                const int e = e0 + u * NT;
                if (e >= ncoef) break;
                const int i = gi[u];
                if (!FEWHA_IN(off + gix[e], I.N, 1, kDbgCoef)) continue;
                const float z = vj[u] * vr[u];
                const float sv = Zc[e] + va[u] * z;
                const float pv = (k == 0) ? z : z + fb * vp[u];
                const float qv = (k == 0) ? sv : sv + fb * vq[u];
                const float cv = vc[u] + fa * pv;
                const float rv = vr[u] - fa * qv;
                if (st) {   // the frame's later iterations read them here; c, r persist from the last
                    st[e] = rv;
                    st[sts + e] = pv;
                    st[2 * sts + e] = qv;
                    st[3 * sts + e] = cv;
                    if (last) {
                        I.c[i] = cv;
                        I.r[i] = rv;
                    }
                } else {
                    I.p[i] = pv;
                    I.q[i] = qv;
                    I.c[i] = cv;
                    I.r[i] = rv;
                }
                float zout;
                if (!last) {
                    zout = vj[u] * rv;
                    rho_p.add_prod(rv, zout);
                    dz_p.add_prod3(va[u], zout, zout);
                } else {
                    zout = cv;
                }
                Zc[e] = zout;
            }
        }
    }
    if (mode != kLpIter) {
        for (int e = tid; e < ncoef; e += NT) {
            const int i = off + gix[e];
            if (!FEWHA_IN(i, I.N, 1, kDbgCoef)) continue;
            const float jinv = __ldg(I.Jinv + i), ad = __ldg(I.aD + i);
            float zout = 0.f;
            if (mode == kLpRhsStart) {
                const float bv = Zc[e];
                float rv;
                if (!P.warm) {
                    rv = bv;
                    I.c[i] = 0.f;
                } else {
                    rv = (bv - I.bprev[i]) + I.r[i];
                }
                I.b[i] = bv;
                I.bprev[i] = bv;
                I.r[i] = rv;
                if (st) {
                    st[e] = rv;
                    st[3 * sts + e] = P.warm ? I.c[i] : 0.f;
                    st[4 * sts + e] = jinv;
                    st[5 * sts + e] = ad;
                }
                zout = jinv * rv;
                rho_p.add_prod(rv, zout);
                dz_p.add_prod3(ad, zout, zout);
            } else if (mode == kLpRhsRepl) {
                I.b[i] = Zc[e];
                zout = I.c[i];
            } else if (mode == kLpReplStart) {
                // r = b - M c = W P^T Gamma^T C^{-1} (s - Gamma P W^T c) - alpha D c
                const float cv = I.c[i];
                const float rv = (float)((double)Zc[e] - (double)ad * (double)cv);
                I.bprev[i] = I.b[i];
                I.r[i] = rv;
                if (st) {
                    st[e] = rv;
                    st[3 * sts + e] = cv;
                    st[4 * sts + e] = jinv;
                    st[5 * sts + e] = ad;
                }
                zout = jinv * rv;
                rho_p.add_prod(rv, zout);
                dz_p.add_prod3(ad, zout, zout);
            }
            Zc[e] = zout;
        }
    }
    if (mode == kLpIter) fmark(P, 18);
    if (make_z) {
        // the partials go out after the inverse's cluster barrier, whose
        // release would otherwise wait for this global store
        const float4 rd = block_reduce2(rho_p, dz_p, (float4*)red);
        if (tid == 0) reinterpret_cast<float4*>(red)[31] = rd;
    }

    // ---- inverse W^T -> phi: row synthesis, exchange, column synthesis ----
    fmark(P, 14);
    const bool need_phi = make_z || mode == kLpRhsRepl || (last && P.out_layers);
    if (need_phi) {
        __syncthreads();
        casc_rows_inv(P, tab, Zc, Urow, T, rem[1], n, R, lR);
        fmark(P, 53);
        cl.sync();     // inverse 2. every owner's stores into this CTA's columns of U have landed
        if (make_z && tid == 0) {
            const int par = (mode == kLpIter) ? ((k + 1) & 1) : 0;
            P.lpart[(size_t)par * P.n_litems * C + (size_t)li * C + rank] = reinterpret_cast<const float4*>(red)[31];
        }
        fmark(P, 54);
        casc_cols_inv(P, Ucol, Z, T, n, J, R, lR);
        fmark(P, 15);
        float* dst = I.phi + off + c0;
        if (!FEWHA_IN(off + c0 + (n - 1) * n, I.N, R, kDbgPhiOut)) return;   // after the last cluster barrier
        casc_copy(n, lR, true, [&](int p) { return (const float*)(Z + (p << lR)); }, [&](int p) { return dst + p * n; });
        if (last && P.phi_out) {   // the caller's buffer: 16-byte pieces when it is 16-byte aligned
            float* d2 = P.phi_out + off + c0;
            casc_copy(n, lR, ((unsigned long long)P.phi_out & 15) == 0,
                      [&](int p) { return (const float*)(Z + (p << lR)); }, [&](int p) { return d2 + p * n; });
        }
    }
    fmark(P, 16);
}
