// Solve sweeps of many cavities with one launch per tree level and phase
// across all of them (batched-cavity extension; the paper treats one
// scatterer at a time, its Sec. 7.3 sweep handles all cells of a level
// independently).  The cavities' trees have different depths: the upward
// sweep is aligned from the leaves (step j works on level L_c - j of every
// cavity that still has a level above its top there), the downward sweep
// from the top (step t on level l0_c + 1 + t), and the top solves of all
// cavities are one batched GEMM.  Every phase of a step (Z = A^{-1} R, the
// skeleton copies of V, the T part of V, A~ times U, the placement in the
// parent, and downward the gathers and the two updates) is one launch over
// the cells of all participating cavities, driven by descriptor arrays
// built once per call on the host.  complex128 (FDS_FP64, LU variant) only.
#include <algorithm>
#include <cstring>
#include <memory>
#include <vector>

#include "fds_internal.cuh"
#include "solve.cuh"

namespace {

// child skeleton rows <-> parent DOF rows of one cell (eq. (rhs_rearrangement))
struct PlaceJob {
    cplx *child;         // the cell's skeleton rows (F or Y of its level)
    cplx *parent;        // the parent cell's first DOF row (R or Z of the level above, or the top)
    int64_t ldc, ldp;
    int r, k1, pos1, pos2, pext, nc;
};

// skeleton copies of the structured V (U[skeleton q] = Z[vmap[q]])
struct SkelJob {
    const cplx *src;     // the cell's DOF rows of Z
    cplx *dst;           // the cell's skeleton rows of U
    int64_t lds, ldd;
    const int *vm;       // the cell's permuted DOF order (device)
    int k1, k2, n1, nc;
};

// natural-order right-hand side <-> leaf-order vector of one cavity
struct GatherJob {
    const int *gidx;
    cplx *rhs;
    cplx *vec;
    int64_t D, ldr;
    int nc;
};

struct CopyJob {
    const cplx *src;
    cplx *dst;
    int64_t n;
};

__global__ void k_place_jobs(const PlaceJob *__restrict__ jobs, int dir) {
    const PlaceJob J = jobs[blockIdx.x];
    for (int64_t e = threadIdx.x; e < (int64_t)J.r * J.nc; e += blockDim.x) {
        const int q = (int)(e % J.r);
        const int64_t c = e / J.r;
        const int pr = q < J.k1 ? J.pos1 + q : J.pos2 + (q - J.k1);
        if (!FDS_IN_RANGE(pr, J.pext)) continue;
        if (dir == 0) J.parent[pr + c * J.ldp] = J.child[q + c * J.ldc];
        else J.child[q + c * J.ldc] = J.parent[pr + c * J.ldp];
    }
}

__global__ void k_skel_jobs(const SkelJob *__restrict__ jobs) {
    const SkelJob J = jobs[blockIdx.x];
    const int kt = J.k1 + J.k2;
    for (int64_t e = threadIdx.x; e < (int64_t)kt * J.nc; e += blockDim.x) {
        const int q = (int)(e % kt);
        const int64_t col = e / kt;
        const int c = q < J.k1 ? 0 : 1;
        const int li = J.vm[(c ? J.n1 : 0) + (c ? q - J.k1 : q)];
        J.dst[q + col * J.ldd] = J.src[li + col * J.lds];
    }
}

__global__ void k_gather_jobs(const GatherJob *__restrict__ jobs, int dir) {
    const GatherJob J = jobs[blockIdx.y];
    const int64_t tot = J.D * J.nc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e % J.D, c = e / J.D;
        if (!FDS_IN_RANGE(J.gidx[q], J.ldr)) continue;
        const int64_t g = J.gidx[q] + c * J.ldr;
        if (dir == 0) J.vec[q + c * J.D] = J.rhs[g];
        else J.rhs[g] = J.vec[q + c * J.D];
    }
}

__global__ void k_copy_jobs(const CopyJob *__restrict__ jobs) {
    const CopyJob J = jobs[blockIdx.y];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < J.n; e += (int64_t)gridDim.x * blockDim.x)
        J.dst[e] = J.src[e];
}

// One GEMM phase: C = alpha op(A) B + beta C over the batch.
struct GemmPhase {
    size_t a = 0, b = 0, c = 0, m = 0;   // byte offsets of the descriptor arrays in the plan buffer
    int batch = 0, max_m = 0, max_n = 0;
    bool mapped = false;
};

struct JobPhase {
    size_t off = 0;
    int n = 0;
};

// Host image of the plan's device buffer: arrays appended at 256-byte boundaries.
struct Blob {
    std::vector<unsigned char> bytes;
    template <class T>
    size_t put(const std::vector<T> &v) {
        const size_t off = (bytes.size() + 255) & ~size_t(255);
        bytes.resize(off + std::max<size_t>(v.size(), 1) * sizeof(T));
        if (!v.empty()) std::memcpy(bytes.data() + off, v.data(), v.size() * sizeof(T));
        return off;
    }
};

struct UpStep {
    GemmPhase ainv, vt, at;
    JobPhase skel, place;
};
struct DownStep {
    GemmPhase at, w;
    JobPhase place;
};

struct Plan {
    std::vector<UpStep> up;
    std::vector<DownStep> down;
    GemmPhase top;
    JobPhase copy;
    Blob blob;
    DBuf<unsigned char> dev;
    std::vector<int> nc;                // the chunk shape the descriptors were built for
    cudaGraphExec_t exec = nullptr;     // the captured sweep (use_graph)
    ~Plan() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

MatRef mref(cplx *p, int rows, int cols, int64_t ld) {
    MatRef r;
    r.p = p;
    r.rows = rows;
    r.cols = cols;
    r.ld = (int)std::max<int64_t>(ld, 1);
    return r;
}

template <class T>
const T *at_off(const DBuf<unsigned char> &d, size_t off) {
    return reinterpret_cast<const T *>(d.p + off);
}

// launch one GEMM phase in batches of at most 65535 (the grid's y extent)
int run_gemm(const Plan &P, const GemmPhase &g, cplx alpha, cplx beta, int accumulate, cudaStream_t s) {
    if (g.batch == 0) return FDS_OK;
    const MatRef *A = at_off<MatRef>(P.dev, g.a), *B = at_off<MatRef>(P.dev, g.b), *C = at_off<MatRef>(P.dev, g.c);
    const RowMaps *M = g.mapped ? at_off<RowMaps>(P.dev, g.m) : nullptr;
    for (int b0 = 0; b0 < g.batch; b0 += 65535) {
        const int nb = std::min(65535, g.batch - b0);
        if (g.mapped)
            FDS_TRY(dense_gemm_map(nb, std::max(g.max_m, 1), g.max_n, A + b0, 0, B + b0, C + b0, M + b0, accumulate, s));
        else
            FDS_TRY(dense_gemm(nb, std::max(g.max_m, 1), g.max_n, A + b0, 0, B + b0, 0, C + b0, alpha, beta, s));
    }
    return FDS_OK;
}

int run_jobs(const Plan &P, const JobPhase &j, int kind, int dir, cudaStream_t s) {
    if (j.n == 0) return FDS_OK;
    for (int b0 = 0; b0 < j.n; b0 += 65535) {
        const int nb = std::min(65535, j.n - b0);
        switch (kind) {
            case 0:
                fds_count_launch(), k_place_jobs<<<nb, 256, 0, s>>>(at_off<PlaceJob>(P.dev, j.off) + b0, dir);
                break;
            case 1:
                fds_count_launch(), k_skel_jobs<<<nb, 256, 0, s>>>(at_off<SkelJob>(P.dev, j.off) + b0);
                break;
            default:
                fds_count_launch(), k_copy_jobs<<<dim3(64, nb), 256, 0, s>>>(at_off<CopyJob>(P.dev, j.off) + b0);
                break;
        }
        FDS_CUDA_TRY(cudaGetLastError());
    }
    return FDS_OK;
}

// The sweep plan of a column chunk in which cavity i solves nc[i] columns (0: idle).
int build_plan(Plan &P, fds_handle *const *h, int count, const std::vector<int> &nc) {
    P.nc = nc;
    int maxup = 0;
    for (int i = 0; i < count; ++i)
        if (nc[i] > 0) maxup = std::max(maxup, h[i]->L - h[i]->l0);
    Blob &B = P.blob;
    P.up.assign(maxup, UpStep());
    P.down.assign(maxup, DownStep());
    for (int j = 0; j < maxup; ++j) {
        std::vector<MatRef> aA, aB, aC, vA, vB, vC, tA, tB, tC;
        std::vector<RowMaps> vM;
        std::vector<SkelJob> sk;
        std::vector<PlaceJob> pl;
        UpStep &U = P.up[j];
        for (int i = 0; i < count; ++i) {
            fds_handle *H = h[i];
            const int l = H->L - j;
            if (nc[i] == 0 || l <= H->l0) continue;
            const Level &C = H->lv[l];
            const Level &Pn = H->lv[l - 1];
            const int64_t D = C.D, R = std::max<int64_t>(C.Rtot, 1);
            cplx *Rv = H->wr[l].p, *Z = H->wz[l].p, *F = H->wf[l].p, *Uv = H->wt[l].p;
            cplx *par = (l - 1 > H->l0) ? H->wr[l - 1].p : H->wtop.p;
            const int64_t ldp = (l - 1 > H->l0) ? Pn.D : std::max<int64_t>(H->Dtop, 1);
            for (int b = 0; b < C.nb; ++b) {
                const int d = C.n1[b] + C.n2[b], r = C.k1[b] + C.k2[b];
                aA.push_back(mref(C.Ainv.p + C.offA[b], d, d, d));
                aB.push_back(mref(Rv + C.doff[b], d, nc[i], D));
                aC.push_back(mref(Z + C.doff[b], d, nc[i], D));
                U.ainv.max_m = std::max(U.ainv.max_m, d);
                SkelJob s{Z + C.doff[b], Uv + C.roff[b], D, R, C.d_vmap.p + C.doff[b], C.k1[b], C.k2[b], C.n1[b],
                          nc[i]};
                sk.push_back(s);
                for (int c = 0; c < 2; ++c) {
                    const int n = c ? C.n2[b] : C.n1[b], k = c ? C.k2[b] : C.k1[b], m = n - k;
                    const int coff = c ? C.n1[b] : 0;
                    vA.push_back(mref(C.T.p + C.toff_h[2 * b + c], k, m, k));
                    vB.push_back(mref(Z + C.doff[b], d, nc[i], D));
                    vC.push_back(mref(Uv + C.roff[b] + (c ? C.k1[b] : 0), k, nc[i], R));
                    RowMaps mp;
                    mp.b = C.d_vmap.p + C.doff[b] + coff + k;
                    mp.c = nullptr;
                    mp.cext = 0;
                    vM.push_back(mp);
                    U.vt.max_m = std::max(U.vt.max_m, k);
                }
                tA.push_back(mref(C.At.p + C.offAt[b], r, r, r));
                tB.push_back(mref(Uv + C.roff[b], r, nc[i], R));
                tC.push_back(mref(F + C.roff[b], r, nc[i], R));
                U.at.max_m = std::max(U.at.max_m, r);
                const int pb = b >> 1;
                PlaceJob p{F + C.roff[b], par + Pn.doff[pb], R, ldp, r, C.k1[b], C.par_pos1[b], C.par_pos2[b],
                           (int)(Pn.doff[pb + 1] - Pn.doff[pb]), nc[i]};
                if (l - 1 == H->l0) p.pext = Pn.n1[pb] + Pn.n2[pb];
                pl.push_back(p);
            }
            U.ainv.max_n = U.vt.max_n = U.at.max_n = std::max(U.ainv.max_n, nc[i]);
        }
        U.ainv.batch = (int)aA.size();
        U.ainv.a = B.put(aA); U.ainv.b = B.put(aB); U.ainv.c = B.put(aC);
        U.vt.batch = (int)vA.size();
        U.vt.a = B.put(vA); U.vt.b = B.put(vB); U.vt.c = B.put(vC); U.vt.m = B.put(vM);
        U.vt.mapped = true;
        U.at.batch = (int)tA.size();
        U.at.a = B.put(tA); U.at.b = B.put(tB); U.at.c = B.put(tC);
        U.skel.off = B.put(sk); U.skel.n = (int)sk.size();
        U.place.off = B.put(pl); U.place.n = (int)pl.size();
    }
    // top solves (x_top = A_top^{-1} f_top) and the copy back into the top vector
    {
        std::vector<MatRef> A, Bv, C;
        std::vector<CopyJob> cp;
        for (int i = 0; i < count; ++i) {
            fds_handle *H = h[i];
            if (nc[i] == 0) continue;
            const int64_t ldt = std::max<int64_t>(H->Dtop, 1);
            A.push_back(mref(H->Atop_inv.p, (int)H->Dtop, (int)H->Dtop, ldt));
            Bv.push_back(mref(H->wtop.p, (int)H->Dtop, nc[i], ldt));
            C.push_back(mref(H->wtop2.p, (int)H->Dtop, nc[i], ldt));
            P.top.max_m = std::max<int>(P.top.max_m, (int)H->Dtop);
            P.top.max_n = std::max(P.top.max_n, nc[i]);
            cp.push_back(CopyJob{H->wtop2.p, H->wtop.p, ldt * nc[i]});
        }
        P.top.batch = (int)A.size();
        P.top.a = B.put(A); P.top.b = B.put(Bv); P.top.c = B.put(C);
        P.copy.off = B.put(cp); P.copy.n = (int)cp.size();
    }
    for (int t = 0; t < maxup; ++t) {
        std::vector<MatRef> aA, aB, aC, wA, wB, wC;
        std::vector<PlaceJob> pl;
        DownStep &Dn = P.down[t];
        for (int i = 0; i < count; ++i) {
            fds_handle *H = h[i];
            const int l = H->l0 + 1 + t;
            if (nc[i] == 0 || l > H->L) continue;
            const Level &C = H->lv[l];
            const Level &Pn = H->lv[l - 1];
            const int64_t D = C.D, R = std::max<int64_t>(C.Rtot, 1);
            cplx *Z = H->wz[l].p, *F = H->wf[l].p, *Y = H->wt[l].p;
            cplx *par = (l - 1 > H->l0) ? H->wz[l - 1].p : H->wtop.p;
            const int64_t ldp = (l - 1 > H->l0) ? Pn.D : std::max<int64_t>(H->Dtop, 1);
            for (int b = 0; b < C.nb; ++b) {
                const int d = C.n1[b] + C.n2[b], r = C.k1[b] + C.k2[b];
                const int pb = b >> 1;
                PlaceJob p{Y + C.roff[b], par + Pn.doff[pb], R, ldp, r, C.k1[b], C.par_pos1[b], C.par_pos2[b],
                           (int)(Pn.doff[pb + 1] - Pn.doff[pb]), nc[i]};
                if (l - 1 == H->l0) p.pext = Pn.n1[pb] + Pn.n2[pb];
                pl.push_back(p);
                aA.push_back(mref(C.At.p + C.offAt[b], r, r, r));
                aB.push_back(mref(Y + C.roff[b], r, nc[i], R));
                aC.push_back(mref(F + C.roff[b], r, nc[i], R));
                Dn.at.max_m = std::max(Dn.at.max_m, r);
                wA.push_back(mref(C.W.p + C.offW[b], d, r, d));
                wB.push_back(mref(F + C.roff[b], r, nc[i], R));
                wC.push_back(mref(Z + C.doff[b], d, nc[i], D));
                Dn.w.max_m = std::max(Dn.w.max_m, d);
            }
            Dn.at.max_n = Dn.w.max_n = std::max(Dn.at.max_n, nc[i]);
        }
        Dn.place.off = B.put(pl); Dn.place.n = (int)pl.size();
        Dn.at.batch = (int)aA.size();
        Dn.at.a = B.put(aA); Dn.at.b = B.put(aB); Dn.at.c = B.put(aC);
        Dn.w.batch = (int)wA.size();
        Dn.w.a = B.put(wA); Dn.w.b = B.put(wB); Dn.w.c = B.put(wC);
    }
    return FDS_OK;
}

// right-hand sides <-> leaf vectors of a chunk: dir 0 into R of the leaf
// level, dir 1 from Z
std::vector<GatherJob> gather_jobs(fds_handle *const *h, int count, const std::vector<int> &nc,
                                   double *const *d_rhs, int c0, int dir) {
    std::vector<GatherJob> g;
    for (int i = 0; i < count; ++i) {
        fds_handle *H = h[i];
        if (nc[i] == 0) continue;
        const int64_t ld = 2LL * H->N;
        g.push_back(GatherJob{H->d_leaf_gidx.p, reinterpret_cast<cplx *>(d_rhs[i]) + (int64_t)c0 * ld,
                              dir == 0 ? H->wr[H->L].p : H->wz[H->L].p, H->lv[H->L].D, ld, nc[i]});
    }
    return g;
}

int run_gather(const DBuf<GatherJob> &g, int dir, cudaStream_t s) {
    for (int b0 = 0; b0 < (int)g.n; b0 += 65535) {
        const int nb = std::min(65535, (int)g.n - b0);
        fds_count_launch(), k_gather_jobs<<<dim3(256, nb), 256, 0, s>>>(g.p + b0, dir);
        FDS_CUDA_TRY(cudaGetLastError());
    }
    return FDS_OK;
}

int run_sweep(const Plan &P, cudaStream_t s) {
    const cplx one = mkc(1, 0), zero = mkc(0, 0), mone = mkc(-1, 0);
    for (const UpStep &U : P.up) {
        FDS_TRY(run_gemm(P, U.ainv, one, zero, 0, s));      // Z = A^{-1} R
        FDS_TRY(run_jobs(P, U.skel, 1, 0, s));              // U[skeleton] = Z[skeleton DOFs]
        FDS_TRY(run_gemm(P, U.vt, one, zero, 1, s));        // U[k rows] += T Z[other DOFs]
        FDS_TRY(run_gemm(P, U.at, one, zero, 0, s));        // F = A~ U
        FDS_TRY(run_jobs(P, U.place, 0, 0, s));             // parent R[pos] = F
    }
    FDS_TRY(run_gemm(P, P.top, one, zero, 0, s));           // x_top = A_top^{-1} f_top
    FDS_TRY(run_jobs(P, P.copy, 3, 0, s));
    for (const DownStep &Dn : P.down) {
        FDS_TRY(run_jobs(P, Dn.place, 0, 1, s));            // Y = parent Z[pos]
        FDS_TRY(run_gemm(P, Dn.at, mone, one, 0, s));       // F -= A~ Y
        FDS_TRY(run_gemm(P, Dn.w, mone, one, 0, s));        // Z -= W F
    }
    return FDS_OK;
}

}  // namespace

extern "C" int fds_solve_batch_levels(int32_t count, fds_handle *const *h, double *const *d_rhs,
                                      const int32_t *nrhs, int32_t use_graph, uint64_t stream) {
    if (count < 0) return FDS_ERR_ARG;
    if (count == 0) return FDS_OK;
    if (!h || !d_rhs || !nrhs) return FDS_ERR_ARG;
    int maxrhs = 0;
    for (int i = 0; i < count; ++i) {
        if (!h[i] || nrhs[i] < 0 || (nrhs[i] > 0 && !d_rhs[i])) return FDS_ERR_ARG;
        if (h[i]->opt.precision != FDS_FP64 || h[i]->opt.variant != FDS_VARIANT_LU || h[i]->L == h[i]->l0)
            return FDS_ERR_ARG;
        maxrhs = std::max(maxrhs, (int)nrhs[i]);
    }
    cudaStream_t s = (cudaStream_t)stream;
    // earlier work of every cavity on its own stream has finished
    for (int i = 0; i < count; ++i) FDS_CUDA_TRY(cudaStreamSynchronize(h[i]->stream));
    for (int i = 0; i < count; ++i)
        if (nrhs[i] > 0) FDS_TRY(sweep_workspace(h[i], std::min((int)nrhs[i], SOLVE_CHUNK)));
    FDS_CUDA_TRY(cudaDeviceSynchronize());
    // one plan per chunk shape (all full chunks share one), built and
    // uploaded once; with use_graph its sweep is captured on first use and
    // replayed for the later chunks of the same shape
    std::vector<std::unique_ptr<Plan>> plans;
    int rc = FDS_OK;
    for (int c0 = 0; c0 < maxrhs && rc == FDS_OK; c0 += SOLVE_CHUNK) {
        std::vector<int> nc(count);
        for (int i = 0; i < count; ++i) nc[i] = std::max(0, std::min(SOLVE_CHUNK, (int)nrhs[i] - c0));
        Plan *P = nullptr;
        for (auto &q : plans)
            if (q->nc == nc) P = q.get();
        if (!P) {
            plans.emplace_back(new Plan());
            P = plans.back().get();
            FDS_TRY(build_plan(*P, h, count, nc));
            FDS_TRY(P->dev.upload(P->blob.bytes, s));
        }
        DBuf<GatherJob> gin, gout;
        FDS_TRY(gin.upload(gather_jobs(h, count, nc, d_rhs, c0, 0), s));
        FDS_TRY(gout.upload(gather_jobs(h, count, nc, d_rhs, c0, 1), s));
        FDS_TRY(run_gather(gin, 0, s));
        if (use_graph && s != 0 && !P->exec) {
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const int r = run_sweep(*P, s);
                const cudaError_t e = cudaStreamEndCapture(s, &g);
                if (!(r == FDS_OK && e == cudaSuccess && g && cudaGraphInstantiate(&P->exec, g, 0) == cudaSuccess))
                    P->exec = nullptr;
                if (g) cudaGraphDestroy(g);
            }
            cudaGetLastError();
        }
        if (P->exec) {
            fds_count_launch();
            if (cudaGraphLaunch(P->exec, s) != cudaSuccess) rc = FDS_ERR_CUDA;
        } else {
            rc = run_sweep(*P, s);
        }
        if (rc != FDS_OK) break;
        FDS_TRY(run_gather(gout, 1, s));
        FDS_CUDA_TRY(cudaStreamSynchronize(s));   // the chunk's gather descriptors are freed next
    }
    if (rc != FDS_OK) return rc;
    FDS_CUDA_TRY(cudaStreamSynchronize(s));
    return FDS_OK;
}
