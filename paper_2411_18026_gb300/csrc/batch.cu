// Batched builds and solves of many independent cavities (extension beyond
// the paper, whose runs treat one scatterer at a time).  Each cavity gets its
// own handle and its own library-owned stream; n_streams host threads take
// cavities largest first, so the per-level launches of different cavities
// run concurrently on the GPU, and allocations inside a worker are ordered on
// the cavity's stream (no device-wide synchronisation between cavities).
#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "fds_internal.cuh"

int fds_build_owned(const fds_geometry *g, double omega, double lambda, double mu, double tol,
                    const fds_options *opt, cudaStream_t owned, fds_handle **out);

namespace {

template <class F>
int run_workers(int count, int n_streams, const std::vector<int> &order, F &&job) {
    int dev = 0;
    FDS_CUDA_TRY(cudaGetDevice(&dev));
    std::atomic<int> next{0};
    std::vector<int> rc(count, FDS_OK);
    std::vector<std::string> why(count);
    auto work = [&]() {
        if (cudaSetDevice(dev) != cudaSuccess) return;
        for (int k = next.fetch_add(1); k < count; k = next.fetch_add(1)) {
            const int i = order[k];
            rc[i] = job(i);
            if (rc[i] != FDS_OK) why[i] = fds_last_error_detail();
        }
    };
    const int nt = std::max(1, std::min(n_streams, count));
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(work);
    work();
    for (auto &t : th) t.join();
    for (int i = 0; i < count; ++i)
        if (rc[i] != FDS_OK) {
            fds_set_error_detail(why[i].c_str());   // the worker's detail, for the caller's thread
            return rc[i];
        }
    return FDS_OK;
}

}  // namespace

extern "C" int fds_build_batch(int32_t count, const fds_geometry *g, const double *omega, double lambda, double mu,
                               double tol, const fds_options *opt, int32_t n_streams, fds_handle **out) {
    if (count < 0 || n_streams < 1 || n_streams > 64) return FDS_ERR_ARG;
    if (count == 0) return FDS_OK;
    if (!g || !omega || !out) return FDS_ERR_ARG;
    for (int i = 0; i < count; ++i) out[i] = nullptr;
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return g[a].n_nodes > g[b].n_nodes; });
    const int rc = run_workers(count, n_streams, order, [&](int i) -> int {
        cudaStream_t s = 0;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return FDS_ERR_CUDA;
        AllocStreamScope as(s);
        return fds_build_owned(&g[i], omega[i], lambda, mu, tol, opt, s, &out[i]);
    });
    if (rc != FDS_OK) {
        for (int i = 0; i < count; ++i) {
            fds_destroy(out[i]);
            out[i] = nullptr;
        }
    }
    return rc;
}

extern "C" int fds_solve_batch(int32_t count, fds_handle *const *h, double *const *d_rhs, const int32_t *nrhs,
                               int32_t n_streams) {
    if (count < 0 || n_streams < 1 || n_streams > 64) return FDS_ERR_ARG;
    if (count == 0) return FDS_OK;
    if (!h || !d_rhs || !nrhs) return FDS_ERR_ARG;
    for (int i = 0; i < count; ++i)
        if (!h[i] || nrhs[i] < 0 || (nrhs[i] > 0 && !d_rhs[i])) return FDS_ERR_ARG;
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return (int64_t)h[a]->N * nrhs[a] > (int64_t)h[b]->N * nrhs[b]; });
    int rc = run_workers(count, n_streams, order, [&](int i) -> int {
        if (nrhs[i] == 0) return FDS_OK;
        // solve workspaces are allocated on the handle's own stream when it has one
        AllocStreamScope as(h[i]->owned.s);
        return fds_solve_impl(h[i], (cplx *)d_rhs[i], nrhs[i], h[i]->stream);
    });
    for (int i = 0; i < count; ++i) cudaStreamSynchronize(h[i]->stream);
    return rc;
}

extern "C" uint64_t fds_handle_stream(const fds_handle *h) { return h ? (uint64_t)h->stream : 0; }
