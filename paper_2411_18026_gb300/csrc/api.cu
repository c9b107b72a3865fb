// C ABI of the solver (include/fds.h): argument checks, handle lifetime,
// host<->device copies for the host-buffer entry points.
#include <algorithm>
#include <cmath>
#include <vector>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "fds_internal.cuh"
#include "fw_tc.cuh"

thread_local cudaStream_t g_alloc_stream = 0;
thread_local int g_c64_tensor = 1;

extern "C" void fds_default_options(fds_options *o) {
    if (!o) return;
    o->leaf_size = 64;
    o->proxy_ratio = 1.5;
    o->proxy_points = 64;
    o->top_level = 1;
    o->tol_decay = 0.5;
    o->variant = FDS_VARIANT_LU;
    o->use_graph = 0;
    o->fw_engine = FDS_FW_FF;
    o->merge_c64_levels = 0;
    o->precision = FDS_FP64;
    o->alpha_re = 0.0;
    o->alpha_im = 0.0;
    o->alpha_set = 0;
    o->cuda_stream = 0;
    o->ir_tol = 1e-9;
    o->ir_max_iter = 10;
    o->ir_apply = FDS_APPLY_FF;
    o->sweep_fp64_levels = -1;
    o->sweep_ff = 1;
    o->merge_c64 = 0;
    o->rank_mode = FDS_RANK_ADAPTIVE;
    o->mlp_params = nullptr;
    o->sketch_extra = 12;
    o->record_features = 0;
    o->c64_engine = FDS_C64_SIMT;
}

extern "C" const char *fds_error_string(int code) {
    switch (code) {
        case FDS_OK: return "ok";
        case FDS_ERR_ARG: return "invalid argument";
        case FDS_ERR_CUDA: return "CUDA runtime error";
        case FDS_ERR_OOM: return "device out of memory";
        case FDS_ERR_SINGULAR: return "singular or non-finite pivot";
        case FDS_ERR_NOT_CONVERGED: return "iterative refinement did not converge";
        case FDS_ERR_TIMEOUT: return "device wait budget exceeded";
        case FDS_ERR_STATE: return "handle not ready";
        default: return "unknown error";
    }
}

// Build one handle; owned != 0: the handle takes ownership of that stream and
// runs on it (batched builds), otherwise it runs on opt->cuda_stream.
void fault_from_env();

int fds_build_owned(const fds_geometry *g, double omega, double lambda, double mu, double tol,
                    const fds_options *opt, cudaStream_t owned, fds_handle **out) {
    fault_from_env();
    // the stream is owned from here on: destroyed on every early return
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() {
            if (s) cudaStreamDestroy(s);
        }
    } guard{owned};
    if (!out) return FDS_ERR_ARG;
    *out = nullptr;
    if (!g || !g->xy || g->n_nodes < 8) return FDS_ERR_ARG;
    if (!(omega > 0) || !(mu > 0) || !(lambda + 2.0 * mu > 0) || !(tol >= 0.0 && tol < 1.0)) return FDS_ERR_ARG;
    fds_options o;
    if (opt) o = *opt;
    else fds_default_options(&o);
    if (o.leaf_size < 2 || !(o.proxy_ratio > 1.0) || o.proxy_points < 8 || o.top_level < -64 ||
        (o.precision != FDS_FP64 && o.precision != FDS_MIXED) || !(o.ir_tol >= 0.0) || o.ir_max_iter < 0 ||
        o.ir_max_iter > 100 || (o.ir_apply != FDS_APPLY_FF && o.ir_apply != FDS_APPLY_FP64) ||
        (o.rank_mode != FDS_RANK_ADAPTIVE && o.rank_mode != FDS_RANK_LEARNED) ||
        (o.rank_mode == FDS_RANK_LEARNED && !o.mlp_params) || o.sketch_extra < 1 || o.sketch_extra > 64 || o.sweep_fp64_levels < -1 || o.sweep_ff < 0 ||
        o.sweep_ff > 2 || (o.c64_engine != FDS_C64_SIMT && o.c64_engine != FDS_C64_TENSOR) ||
        !(o.tol_decay > 0.0 && o.tol_decay <= 1.0) ||
        (o.variant != FDS_VARIANT_LU && o.variant != FDS_VARIANT_MR2005) ||
        (o.variant == FDS_VARIANT_MR2005 && o.precision != FDS_FP64) ||
        (o.fw_engine != FDS_FW_FF && o.fw_engine != FDS_FW_TENSOR) || o.merge_c64_levels < 0)
        return FDS_ERR_ARG;
    for (int i = 0; i < 2 * g->n_nodes; ++i)
        if (!std::isfinite(g->xy[i])) return FDS_ERR_ARG;
    // the tree must fit the launch grid (cells per level <= 65535)
    {
        int L = 0;
        while (((g->n_nodes + (1 << L) - 1) >> L) > o.leaf_size) ++L;
        if (L > 15) return FDS_ERR_ARG;
    }
    fds_handle *h = new (std::nothrow) fds_handle();
    if (!h) return FDS_ERR_OOM;
    h->owned.s = owned;
    guard.s = 0;
    h->N = g->n_nodes;
    h->xy.assign(g->xy, g->xy + 2 * (size_t)g->n_nodes);
    h->ph.lambda = lambda;
    h->ph.mu = mu;
    h->ph.rho = g->rho > 0 ? g->rho : 1.0;
    h->ph.omega = omega;
    h->ph.alpha_re = o.alpha_re;
    h->ph.alpha_im = o.alpha_im;
    h->ph.alpha_set = o.alpha_set;
    h->P = make_physdev(&h->ph);
    h->tol = tol;
    h->opt = o;
    h->stream = owned ? owned : (cudaStream_t)o.cuda_stream;
    if (owned) h->opt.cuda_stream = (uint64_t)owned;
    if (o.rank_mode == FDS_RANK_LEARNED) {
        for (int i = 0; i < FDS_MLP_NPARAM; ++i)
            if (!std::isfinite(o.mlp_params[i])) {
                delete h;
                return FDS_ERR_ARG;
            }
        std::vector<float> prm(o.mlp_params, o.mlp_params + FDS_MLP_NPARAM);
        int rc0 = h->d_mlp.upload(prm, h->stream);
        if (rc0 != FDS_OK) {
            delete h;
            return rc0;
        }
    }
    h->opt.mlp_params = nullptr;   // not kept past the call
    int rc = fds_build_impl(h);
    if (rc != FDS_OK) {
        cudaStreamSynchronize(h->stream);
        delete h;
        return rc;
    }
    *out = h;
    return FDS_OK;
}

extern "C" int fds_build_ex(const fds_geometry *g, double omega, double lambda, double mu, double tol,
                            const fds_options *opt, fds_handle **out) {
    return fds_build_owned(g, omega, lambda, mu, tol, opt, 0, out);
}

extern "C" int fds_build(const fds_geometry *g, double omega, double lambda, double mu, double tol,
                         fds_handle **out) {
    return fds_build_ex(g, omega, lambda, mu, tol, nullptr, out);
}

extern "C" int fds_rhs_plane_wave_device(fds_handle *h, const int32_t *d_kinds, const double *d_angles,
                                         int32_t nrhs, double *d_f, uint64_t stream) {
    if (!h || nrhs < 0) return FDS_ERR_ARG;
    if (nrhs == 0) return FDS_OK;
    if (!d_kinds || !d_angles || !d_f) return FDS_ERR_ARG;
    return fds_rhs_impl(h, d_kinds, d_angles, nrhs, (cplx *)d_f, (cudaStream_t)stream);
}

extern "C" int fds_rhs_plane_wave(fds_handle *h, const int32_t *kinds, const double *angles, int32_t nrhs,
                                  double *f_out) {
    if (!h || nrhs < 0) return FDS_ERR_ARG;
    if (nrhs == 0) return FDS_OK;
    if (!kinds || !angles || !f_out) return FDS_ERR_ARG;
    for (int j = 0; j < nrhs; ++j)
        if (kinds[j] != 0 && kinds[j] != 1) return FDS_ERR_ARG;
    cudaStream_t s = h->stream;
    DBuf<int> dk;
    DBuf<double> da;
    DBuf<cplx> df;
    FDS_TRY(dk.alloc(nrhs));
    FDS_TRY(da.alloc(nrhs));
    FDS_TRY(df.alloc((size_t)2 * h->N * nrhs));
    FDS_CUDA_TRY(cudaMemcpyAsync(dk.p, kinds, sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
    FDS_CUDA_TRY(cudaMemcpyAsync(da.p, angles, sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    FDS_TRY(fds_rhs_impl(h, dk.p, da.p, nrhs, df.p, s));
    FDS_CUDA_TRY(cudaMemcpyAsync(f_out, df.p, sizeof(cplx) * 2 * h->N * nrhs, cudaMemcpyDeviceToHost, s));
    FDS_CUDA_TRY(cudaStreamSynchronize(s));
    return FDS_OK;
}

extern "C" int fds_solve_device(fds_handle *h, double *d_rhs, int32_t nrhs, uint64_t stream) {
    if (!h || nrhs < 0) return FDS_ERR_ARG;
    if (nrhs == 0) return FDS_OK;
    if (!d_rhs) return FDS_ERR_ARG;
    return fds_solve_impl(h, (cplx *)d_rhs, nrhs, (cudaStream_t)stream);
}

// Host buffers: column chunks of the right-hand sides stream through two
// device buffers; the copies of the next chunk in and of the previous chunk
// out run on a second stream while the handle's stream solves the current
// chunk (they overlap when the host memory is page-locked).
namespace {
constexpr int SOLVE_CHUNK_HOST = 256;   // right-hand sides per host-buffer chunk
struct CopyPipe {
    cudaStream_t c = nullptr;
    cudaEvent_t in[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr};
    ~CopyPipe() {
        if (c) cudaStreamSynchronize(c);
        for (int q = 0; q < 2; ++q) {
            if (in[q]) cudaEventDestroy(in[q]);
            if (done[q]) cudaEventDestroy(done[q]);
        }
        if (c) cudaStreamDestroy(c);
    }
};
}  // namespace

extern "C" int fds_solve(fds_handle *h, double *rhs, int32_t nrhs) {
    if (!h || nrhs < 0) return FDS_ERR_ARG;
    if (nrhs == 0) return FDS_OK;
    if (!rhs) return FDS_ERR_ARG;
    cudaStream_t s = h->stream;
    const int64_t ld = 2LL * h->N;
    const int chunk = std::min<int>(nrhs, SOLVE_CHUNK_HOST);
    const int nch = (nrhs + chunk - 1) / chunk;
    cplx *host = reinterpret_cast<cplx *>(rhs);
    DBuf<cplx> buf[2];
    for (int q = 0; q < std::min(nch, 2); ++q) FDS_TRY(buf[q].alloc((size_t)ld * chunk));
    CopyPipe P;
    FDS_CUDA_TRY(cudaStreamCreateWithFlags(&P.c, cudaStreamNonBlocking));
    for (int q = 0; q < 2; ++q) {
        FDS_CUDA_TRY(cudaEventCreateWithFlags(&P.in[q], cudaEventDisableTiming));
        FDS_CUDA_TRY(cudaEventCreateWithFlags(&P.done[q], cudaEventDisableTiming));
    }
    auto cols = [&](int c) { return std::min(chunk, nrhs - c * chunk); };
    auto copy_in = [&](int c) -> int {
        cplx *d = buf[c & 1].p;
        FDS_CUDA_TRY(cudaMemcpyAsync(d, host + (int64_t)c * chunk * ld, sizeof(cplx) * ld * cols(c),
                                     cudaMemcpyHostToDevice, P.c));
        FDS_CUDA_TRY(cudaEventRecord(P.in[c & 1], P.c));
        return FDS_OK;
    };
    FDS_TRY(copy_in(0));
    if (nch > 1) FDS_TRY(copy_in(1));
    int worst = FDS_OK, iters = 0;
    double ms = 0, res = -1.0;
    for (int c = 0; c < nch; ++c) {
        const int q = c & 1;
        FDS_CUDA_TRY(cudaStreamWaitEvent(s, P.in[q], 0));
        const int rc = fds_solve_impl(h, buf[q].p, cols(c), s);
        if (rc != FDS_OK && rc != FDS_ERR_NOT_CONVERGED) return rc;
        if (rc != FDS_OK) worst = rc;
        ms += h->solve_ms;
        iters = std::max(iters, h->ir_iters);
        res = std::max(res, h->ir_residual);
        FDS_CUDA_TRY(cudaEventRecord(P.done[q], s));
        FDS_CUDA_TRY(cudaStreamWaitEvent(P.c, P.done[q], 0));
        FDS_CUDA_TRY(cudaMemcpyAsync(host + (int64_t)c * chunk * ld, buf[q].p, sizeof(cplx) * ld * cols(c),
                                     cudaMemcpyDeviceToHost, P.c));
        if (c + 2 < nch) FDS_TRY(copy_in(c + 2));
    }
    FDS_CUDA_TRY(cudaStreamSynchronize(P.c));
    h->solve_ms = ms;
    h->ir_iters = iters;
    h->ir_residual = res;
    return worst;
}

extern "C" int fds_stats_get(const fds_handle *h, fds_stats *st) {
    if (!h || !st) return FDS_ERR_ARG;
    *st = fds_stats{};
    st->n_nodes = h->N;
    st->levels = h->L;
    st->top_level = h->l0;
    st->top_size = (int)h->Dtop;
    for (int l = h->l0 + 1; l <= h->L && l < 32; ++l) {
        const Level &C = h->lv[l];
        int64_t sum = 0;
        int mx = 0;
        for (int b = 0; b < C.nb; ++b) {
            sum += C.k1[b] + C.k2[b];
            mx = std::max(mx, C.k1[b] + C.k2[b]);
        }
        st->skeleton_dofs[l] = sum;
        st->max_rank[l] = mx;
    }
    st->build_ms = h->build_ms;
    st->solve_ms = h->solve_ms;
    st->factor_bytes = h->factor_bytes;
    st->ir_iters = h->ir_iters;
    st->ir_residual = h->ir_residual;
    st->id_sketched = h->id_sketched;
    st->id_fallback = h->id_fallback;
    st->features_recorded = (int64_t)h->frac_rows.size();
    return FDS_OK;
}

extern "C" int fds_level_ranks(const fds_handle *h, int32_t level, int32_t *k, int32_t cap) {
    if (!h || !k || level <= h->l0 || level > h->L) return FDS_ERR_ARG;
    const Level &C = h->lv[level];
    if (cap < 2 * C.nb) return FDS_ERR_ARG;
    for (int b = 0; b < C.nb; ++b) {
        k[2 * b] = C.k1[b];
        k[2 * b + 1] = C.k2[b];
    }
    return 2 * C.nb;
}

extern "C" int fds_features_get(const fds_handle *h, float *feat, float *frac, int32_t cap) {
    if (!h || cap < 0 || (cap > 0 && (!feat || !frac))) return FDS_ERR_ARG;
    const int64_t n = std::min<int64_t>(cap, (int64_t)h->frac_rows.size());
    for (int64_t r = 0; r < n; ++r) {
        frac[r] = h->frac_rows[r];
        for (int i = 0; i < FDS_MLP_NIN; ++i) feat[r * FDS_MLP_NIN + i] = h->feat_rows[r * FDS_MLP_NIN + i];
    }
    return (int)n;
}

extern "C" void fds_destroy(fds_handle *h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    delete h;
}

// ------------------------------------------------------------------ fault injection
namespace {
std::atomic<int64_t> g_fault_alloc{0};   // allocations left before the injected failure (0: disarmed)
std::atomic<int> g_fault_nan{0};
std::atomic<int> g_fault_tc_armed{0};    // bit 0: leaf-block product, bit 1: complex64 GEMM
}  // namespace

bool fds_fault_alloc_fires() {
    int64_t v = g_fault_alloc.load(std::memory_order_relaxed);
    while (v > 0)
        if (g_fault_alloc.compare_exchange_weak(v, v - 1)) return v == 1;
    return false;
}

bool fds_fault_nan_fires() { return g_fault_nan.exchange(0) != 0; }

extern "C" int fds_fault_inject(int32_t kind, int64_t arg) {
    switch (kind) {
        case FDS_FAULT_NONE: {
            g_fault_alloc.store(0);
            g_fault_nan.store(0);
            // the device flags are touched only if a stall was armed
            const int armed = g_fault_tc_armed.exchange(0);
            if (armed & 1) FDS_TRY(oz_fault_arm(0));
            if (armed & 2) FDS_TRY(tc_fault_arm(0));
            return FDS_OK;
        }
        case FDS_FAULT_ALLOC:
            if (arg < 1) return FDS_ERR_ARG;
            g_fault_alloc.store(arg);
            return FDS_OK;
        case FDS_FAULT_NAN_BLOCK:
            g_fault_nan.store(1);
            return FDS_OK;
        case FDS_FAULT_TC_STALL_FW:
            FDS_TRY(oz_fault_arm(1));
            g_fault_tc_armed.fetch_or(1);
            return FDS_OK;
        case FDS_FAULT_TC_STALL_C64:
            FDS_TRY(tc_fault_arm(1));
            g_fault_tc_armed.fetch_or(2);
            return FDS_OK;
        default:
            return FDS_ERR_ARG;
    }
}

// FDS_FAULT in the environment (alloc:N, nan, stall_fw, stall_c64) arms that
// fault once per process, at the first build
void fault_from_env() {
    static std::once_flag once;
    std::call_once(once, [] {
        const char *v = std::getenv("FDS_FAULT");
        if (!v) return;
        if (!std::strncmp(v, "alloc:", 6)) {
            const long long n = std::atoll(v + 6);
            if (n >= 1) fds_fault_inject(FDS_FAULT_ALLOC, n);
        } else if (!std::strcmp(v, "nan")) {
            fds_fault_inject(FDS_FAULT_NAN_BLOCK, 0);
        } else if (!std::strcmp(v, "stall_fw")) {
            fds_fault_inject(FDS_FAULT_TC_STALL_FW, 0);
        } else if (!std::strcmp(v, "stall_c64")) {
            fds_fault_inject(FDS_FAULT_TC_STALL_C64, 0);
        }
    });
}

// ------------------------------------------------------------------ bounds-checked build
namespace {
std::vector<unsigned long long (*)()> &bounds_units() {
    static std::vector<unsigned long long (*)()> v;
    return v;
}
}  // namespace

int fds_bounds_register(unsigned long long (*take)()) {
    bounds_units().push_back(take);
    return 1;
}

extern "C" int fds_bounds_violations(int64_t *count) {
#ifdef FDS_CHECKS
    if (!count) return FDS_ERR_ARG;
    FDS_CUDA_TRY(cudaDeviceSynchronize());
    unsigned long long t = 0;
    for (auto f : bounds_units()) t += f();
    *count = (int64_t)t;
    return FDS_OK;
#else
    (void)count;
    return FDS_ERR_STATE;
#endif
}
