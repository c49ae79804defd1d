// C ABI of libfewha.so (declared in include/fewha.h).  Argument checking and
// dispatch only; the work runs in the kernels of solver.cu / fused.cu.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fewha.h"
#include "setup.h"
#include "solver.h"

namespace fewha {
// records of the debug build's bounds checks, one reader per CUDA source
int dbg_read_fused(unsigned long long* first, unsigned long long* count);
int dbg_read_solver(unsigned long long* first, unsigned long long* count);
int dbg_read_fitcg(unsigned long long* first, unsigned long long* count);
int dbg_read_noalloc(unsigned long long* first, unsigned long long* count);
}  // namespace fewha

struct fewha_handle {
    fewha::SolverBase* s = nullptr;
    std::string msg;
};

struct fewha_batch {
    fewha::BatchBase* b = nullptr;
    std::string msg;
};

namespace {
thread_local std::string g_create_error;
thread_local std::string g_batch_error;

int bfail(fewha_batch* b, int code, const std::string& m) {
    b->msg = m;
    return code;
}

int bdone(fewha_batch* b, int st) {
    if (st != FEWHA_OK) b->msg = b->b->err;
    return st;
}

int fail(fewha_handle* h, int code, const std::string& m) {
    if (h) h->msg = m;
    return code;
}

int done(fewha_handle* h, int st) {
    if (st != FEWHA_OK && h && h->s) h->msg = h->s->err;
    return st;
}
}  // namespace

extern "C" {

int fewha_create(const fewha_geometry* geom, const fewha_profile* prof, void* stream, fewha_handle** out) {
    if (!out) return FEWHA_ERR_ARG;
    *out = nullptr;
    if (!geom || !prof) {
        g_create_error = "null geometry or profile";
        return FEWHA_ERR_ARG;
    }
    try {
        fewha::HostSetup hs;
        std::string err;
        int st = fewha::build_setup(*geom, *prof, hs, err);
        if (st) {
            g_create_error = err;
            return st;
        }
        fewha::SolverBase* s = fewha::make_solver(hs, (cudaStream_t)stream, err, st);
        if (!s) {
            g_create_error = err;
            return st ? st : FEWHA_ERR_CUDA;
        }
        fewha_handle* h = new fewha_handle();
        h->s = s;
        *out = h;
        return FEWHA_OK;
    } catch (const std::bad_alloc&) {
        g_create_error = "host out of memory";
        return FEWHA_ERR_ARG;
    } catch (...) {
        g_create_error = "unexpected host exception";
        return FEWHA_ERR_ARG;
    }
}

int fewha_destroy(fewha_handle* h) {
    if (!h) return FEWHA_ERR_ARG;
    delete h->s;
    delete h;
    return FEWHA_OK;
}

const char* fewha_last_error(const fewha_handle* h) {
    if (!h) return g_create_error.c_str();
    return h->msg.c_str();
}

int fewha_sizes(const fewha_handle* h, long* n_coeff, long* n_slopes, long* n_act) {
    if (!h) return FEWHA_ERR_ARG;
    if (n_coeff) *n_coeff = h->s->hs.N;
    if (n_slopes) *n_slopes = h->s->hs.S;
    if (n_act) *n_act = h->s->hs.NA;
    return FEWHA_OK;
}

int fewha_set_path(fewha_handle* h, int path) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    if (path != FEWHA_PATH_PLAIN && path != FEWHA_PATH_FUSED) return fail(h, FEWHA_ERR_ARG, "unknown path");
    if (path == FEWHA_PATH_FUSED && h->s->hs.prec != FEWHA_FP32)
        return fail(h, FEWHA_ERR_ARG, "the fused path is FP32 only");
    if (path == FEWHA_PATH_FUSED && !h->s->fused_available)
        return fail(h, FEWHA_ERR_GEOMETRY, "no fused plan for this geometry: " + h->s->fused_reason);
    h->s->path = path;
    return FEWHA_OK;
}

int fewha_set_residual_replacement(fewha_handle* h, int k_rr) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    if (k_rr < 0) return fail(h, FEWHA_ERR_ARG, "k_rr must be >= 0");
    h->s->k_rr = k_rr;
    return FEWHA_OK;
}

int fewha_set_frame(fewha_handle* h, const void* slopes, int on_device) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    return done(h, h->s->set_frame(slopes, on_device));
}

int fewha_solve(fewha_handle* h, int n_iter, int warm_start) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    return done(h, h->s->solve(n_iter, warm_start));
}

int fewha_fit_dm(fewha_handle* h, double gain, int n_fit, void* dm_out, int on_device) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    return done(h, h->s->fit(gain, n_fit, dm_out, on_device));
}

int fewha_get_layers(fewha_handle* h, void* out, int on_device) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    return done(h, h->s->get_layers(out, on_device));
}

int fewha_get_vector(fewha_handle* h, int which, void* out, int on_device) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    return done(h, h->s->get_vector(which, out, on_device));
}

int fewha_get_state(fewha_handle* h, void* c, void* b, void* r, int on_device) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    return done(h, h->s->get_state(c, b, r, on_device));
}

int fewha_set_state(fewha_handle* h, const void* c, const void* b, const void* r, int on_device, long frame_count) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    if (frame_count < 0) return fail(h, FEWHA_ERR_ARG, "frame_count must be >= 0");
    int st = h->s->set_state(c, b, r, on_device, frame_count);
    if (!st) h->s->have_frame = h->s->have_frame;
    return done(h, st);
}

int fewha_apply_M(fewha_handle* h, const void* x, void* y, int on_device) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    return done(h, h->s->apply_M(x, y, on_device));
}

int fewha_frame(fewha_handle* h, const void* slopes, int n_iter, int warm_start, double gain, int n_fit,
                void* layers_out, void* dm_out, int on_device) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    if (dm_out && (n_fit < 0 || !(gain >= 0.0 && gain <= 1.0)))
        return fail(h, FEWHA_ERR_ARG, "gain must be in [0, 1] and n_fit >= 0");
    return done(h, h->s->frame(slopes, n_iter, warm_start, gain, n_fit, layers_out, dm_out, on_device));
}

int fewha_get_frame_timing(fewha_handle* h, double* out) {
    if (!h || !out) return FEWHA_ERR_ARG;
    return done(h, h->s->get_frame_timing(out));
}

int fewha_operator_dims(fewha_handle* h, int op, long* n_in, long* n_out) {
    if (!h || !n_in || !n_out) return FEWHA_ERR_ARG;
    return done(h, h->s->operator_dims(op, *n_in, *n_out));
}

int fewha_apply_operator(fewha_handle* h, int op, const void* x, void* y, int on_device) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    return done(h, h->s->apply_operator(op, x, y, on_device));
}

int fewha_time_operator(fewha_handle* h, int op, int reps, double* us_per_application) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    return done(h, h->s->time_operator(op, reps, us_per_application));
}

int fewha_sync(fewha_handle* h) {
    if (!h) return FEWHA_ERR_ARG;
    return done(h, h->s->sync());
}

int fewha_set_barrier_budget(fewha_handle* h, long long cycles) {
    if (!h) return FEWHA_ERR_ARG;
    if (cycles < 0) return fail(h, FEWHA_ERR_ARG, "budget must be >= 0");
    h->s->barrier_budget = cycles;
    return FEWHA_OK;
}

int fewha_describe(fewha_handle* h, char* buf, int len) {
    if (!h) return FEWHA_ERR_ARG;
    return done(h, h->s->describe(buf, len));
}

int fewha_set_trace(fewha_handle* h, int on) {
    if (!h) return FEWHA_ERR_ARG;
    return done(h, h->s->set_trace(on));
}

int fewha_get_trace(fewha_handle* h, unsigned long long* out, int max_entries, int* slots, int* grid) {
    if (!h) return FEWHA_ERR_ARG;
    if (!slots || !grid || max_entries < 0) return fail(h, FEWHA_ERR_ARG, "bad trace arguments");
    return done(h, h->s->get_trace(out, max_entries, slots, grid));
}

int fewha_get_fine_trace(fewha_handle* h, unsigned long long* out, int max_entries, int* per_cta, int* grid) {
    if (!h) return FEWHA_ERR_ARG;
    if (!per_cta || !grid || max_entries < 0) return fail(h, FEWHA_ERR_ARG, "bad trace arguments");
    return done(h, h->s->get_fine_trace(out, max_entries, per_cta, grid));
}

int fewha_set_cluster_size(fewha_handle* h, int cluster_size) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    if (cluster_size != 1 && cluster_size != 2 && cluster_size != 4 && cluster_size != 8 && cluster_size != 16)
        return fail(h, FEWHA_ERR_ARG, "cluster size must be 1, 2, 4, 8 or 16");
    return done(h, h->s->set_cluster_size(cluster_size));
}

int fewha_set_layer_transform(fewha_handle* h, int form) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    if (form < -1 || form > 1) return fail(h, FEWHA_ERR_ARG, "layer transform must be -1, 0 or 1");
    return done(h, h->s->set_layer_transform(form));
}

int fewha_autotune(fewha_handle* h, int n_iter, int reps, char* report, int len) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    return done(h, h->s->autotune(n_iter, reps, report, len));
}

int fewha_set_loop(fewha_handle* h, int closed) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    if (closed != 0 && closed != 1) return fail(h, FEWHA_ERR_ARG, "closed must be 0 or 1");
    return done(h, h->s->set_loop(closed));
}

int fewha_set_params(fewha_handle* h, const double* cn2_frac, double alpha, const double* w) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    return done(h, h->s->set_params(cn2_frac, alpha, w));
}

long fewha_tape_bytes(const fewha_handle* h, int n_iter) {
    if (!h || n_iter < 1) return -1;
    return (long)h->s->tape_size(n_iter);
}

int fewha_solve_taped(fewha_handle* h, const void* slopes, int n_iter, void* tape, void* layers_out) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    return done(h, h->s->solve_taped(slopes, n_iter, tape, layers_out));
}

int fewha_backward(fewha_handle* h, const void* slopes, int n_iter, const void* tape, const void* layers_bar,
                   double* grad_cn2, double* grad_alpha, double* grad_w, void* grad_slopes) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    return done(h, h->s->backward(slopes, n_iter, tape, layers_bar, grad_cn2, grad_alpha, grad_w, grad_slopes));
}

long fewha_tape_bytes_batch(const fewha_handle* h, int n_iter, int n_frames) {
    if (!h || n_iter < 1 || n_frames < 1 || n_frames > 65535) return -1;
    return (long)h->s->tape_size_batch(n_iter, n_frames);
}

int fewha_solve_taped_batch(fewha_handle* h, int n_frames, const void* slopes, int n_iter, void* tape,
                            void* layers_out) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    return done(h, h->s->solve_taped_batch(n_frames, slopes, n_iter, tape, layers_out));
}

int fewha_backward_batch(fewha_handle* h, int n_frames, const void* slopes, int n_iter, const void* tape,
                         const void* layers_bar, double* grad_cn2, double* grad_alpha, double* grad_w,
                         void* grad_slopes) {
    if (!h) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    return done(h, h->s->backward_batch(n_frames, slopes, n_iter, tape, layers_bar, grad_cn2, grad_alpha, grad_w,
                                        grad_slopes));
}

int fewha_frame_arm(fewha_handle* h, const void* slopes, int n_iter, int warm_start, void* layers_out, double wait_s) {
    if (!h) return FEWHA_ERR_ARG;
    return done(h, h->s->frame_arm(slopes, n_iter, warm_start, layers_out, wait_s));
}

int fewha_frame_fire(fewha_handle* h) {
    if (!h) return FEWHA_ERR_ARG;
    return done(h, h->s->frame_fire());
}

int fewha_set_host_transfer(fewha_handle* h, int slopes_by_copy) {
    if (!h || (slopes_by_copy != 0 && slopes_by_copy != 1)) return FEWHA_ERR_ARG;
    if (h->s && h->s->is_armed()) return fail(h, FEWHA_ERR_STATE, "a frame is armed: fire it first");
    return done(h, h->s->set_host_transfer(slopes_by_copy));
}

long long fewha_launch_count(const fewha_handle* h) {
    if (!h) return -1;
    return h->s->launches;
}

// ---- batch ----

int fewha_batch_create(int count, const fewha_geometry* geoms, const fewha_profile* profs, void* stream,
                       int max_tile_side, int cluster_size, fewha_batch** out) {
    if (!out) return FEWHA_ERR_ARG;
    *out = nullptr;
    if (count < 1 || !geoms || !profs) {
        g_batch_error = "count must be >= 1 with geometries and profiles";
        return FEWHA_ERR_ARG;
    }
    if (max_tile_side < 0 || (cluster_size != 0 && cluster_size != 1 && cluster_size != 2 && cluster_size != 4 &&
                              cluster_size != 8 && cluster_size != 16)) {
        g_batch_error = "max_tile_side must be >= 0 and cluster_size 0, 1, 2, 4, 8 or 16";
        return FEWHA_ERR_ARG;
    }
    try {
        std::vector<fewha::HostSetup> hss(count);
        for (int i = 0; i < count; ++i) {
            std::string err;
            if (geoms[i].precision != FEWHA_FP32) {
                g_batch_error = "instance " + std::to_string(i) + ": batched instances are FP32 only";
                return FEWHA_ERR_ARG;
            }
            int st = fewha::build_setup(geoms[i], profs[i], hss[i], err);
            if (st) {
                g_batch_error = "instance " + std::to_string(i) + ": " + err;
                return st;
            }
        }
        std::string err;
        int st = FEWHA_OK;
        fewha::BatchBase* b = fewha::make_batch(hss, (cudaStream_t)stream, max_tile_side, cluster_size, err, st);
        if (!b) {
            g_batch_error = err;
            return st ? st : FEWHA_ERR_CUDA;
        }
        fewha_batch* h = new fewha_batch();
        h->b = b;
        *out = h;
        return FEWHA_OK;
    } catch (const std::bad_alloc&) {
        g_batch_error = "host out of memory";
        return FEWHA_ERR_ARG;
    } catch (...) {
        g_batch_error = "unexpected host exception";
        return FEWHA_ERR_ARG;
    }
}

int fewha_batch_destroy(fewha_batch* b) {
    if (!b) return FEWHA_ERR_ARG;
    delete b->b;
    delete b;
    return FEWHA_OK;
}

const char* fewha_batch_last_error(const fewha_batch* b) {
    if (!b) return g_batch_error.c_str();
    return b->msg.c_str();
}

int fewha_batch_sizes(const fewha_batch* b, int* count, long* coeff_off, long* slope_off) {
    if (!b) return FEWHA_ERR_ARG;
    const auto& co = b->b->coeff_off;
    const auto& so = b->b->slope_off;
    if (count) *count = (int)co.size() - 1;
    for (size_t i = 0; i < co.size(); ++i) {
        if (coeff_off) coeff_off[i] = co[i];
        if (slope_off) slope_off[i] = so[i];
    }
    return FEWHA_OK;
}

int fewha_batch_set_residual_replacement(fewha_batch* b, int k_rr) {
    if (!b) return FEWHA_ERR_ARG;
    if (k_rr < 0) return bfail(b, FEWHA_ERR_ARG, "k_rr must be >= 0");
    b->b->k_rr = k_rr;
    return FEWHA_OK;
}

int fewha_batch_frame(fewha_batch* b, const void* slopes, int n_iter, int warm_start, void* layers_out,
                      int on_device) {
    if (!b) return FEWHA_ERR_ARG;
    return bdone(b, b->b->frame(slopes, n_iter, warm_start, layers_out, on_device));
}

int fewha_batch_get_state(fewha_batch* b, int inst, void* c, void* bprev, void* r, int on_device) {
    if (!b) return FEWHA_ERR_ARG;
    return bdone(b, b->b->get_state(inst, c, bprev, r, on_device));
}

int fewha_batch_sync(fewha_batch* b) {
    if (!b) return FEWHA_ERR_ARG;
    return bdone(b, b->b->sync());
}

int fewha_batch_describe(fewha_batch* b, char* buf, int len) {
    if (!b) return FEWHA_ERR_ARG;
    return bdone(b, b->b->describe(buf, len));
}

long long fewha_batch_launch_count(const fewha_batch* b) {
    if (!b) return -1;
    return b->b->launches;
}

int fewha_batch_set_trace(fewha_batch* b, int on) {
    if (!b) return FEWHA_ERR_ARG;
    return bdone(b, b->b->set_trace(on));
}

int fewha_batch_get_fine_trace(fewha_batch* b, unsigned long long* out, int max_entries, int* per_cta, int* grid) {
    if (!b || !per_cta || !grid || max_entries < 0) return FEWHA_ERR_ARG;
    return bdone(b, b->b->get_fine_trace(out, max_entries, per_cta, grid));
}

int fewha_batch_autotune(fewha_batch* b, int n_iter, int reps, char* report, int len) {
    if (!b) return FEWHA_ERR_ARG;
    return bdone(b, b->b->autotune(n_iter, reps, report, len));
}

int fewha_batch_set_groups(fewha_batch* b, const int* group, int count) {
    if (!b) return FEWHA_ERR_ARG;
    return bdone(b, b->b->set_groups(group, count));
}

int fewha_batch_set_max_launches(fewha_batch* b, int max_launches) {
    if (!b) return FEWHA_ERR_ARG;
    if (max_launches < 0) {
        b->msg = "max_launches must be >= 0";
        return FEWHA_ERR_ARG;
    }
    b->b->max_launches = max_launches;
    return FEWHA_OK;
}

int fewha_debug_bounds(unsigned long long* first, unsigned long long* count) {
    if (!first || !count) return FEWHA_ERR_ARG;
    int (*const readers[])(unsigned long long*, unsigned long long*) = {
        fewha::dbg_read_fused, fewha::dbg_read_solver, fewha::dbg_read_fitcg, fewha::dbg_read_noalloc};
    *first = 0ull;
    *count = 0ull;
    int built = 0;
    for (auto rd : readers) {
        unsigned long long f = 0ull, c = 0ull;
        const int st = rd(&f, &c);
        if (st < 0) {
            cudaGetLastError();
            return FEWHA_ERR_CUDA;
        }
        built = st;
        if (!*first) *first = f;
        *count += c;
    }
    return built;
}

}  // extern "C"
