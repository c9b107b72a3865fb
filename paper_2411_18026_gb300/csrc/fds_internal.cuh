// Internal state of a factorisation handle (host planner + device buffers).
#pragma once

#include <vector>

#include "common.cuh"
#include "dense.cuh"

// Stream that DBuf allocations of the calling thread are ordered on.  0 (the
// default): plain cudaMalloc / cudaFree.  A batched build sets it, per worker
// thread, to the stream its handle owns: allocation and release are then
// stream-ordered (cudaMallocAsync / cudaFreeAsync), so concurrent builds on
// different streams do not synchronise the device at every release; the
// owned stream outlives every buffer of the handle.
extern thread_local cudaStream_t g_alloc_stream;
// complex64 GEMMs of this thread on the tensor cores (1) or FP32 FMA (0)
extern thread_local int g_c64_tensor;
struct C64EngineScope {
    int prev;
    explicit C64EngineScope(int v) : prev(g_c64_tensor) { g_c64_tensor = v; }
    ~C64EngineScope() { g_c64_tensor = prev; }
};

struct AllocStreamScope {
    cudaStream_t prev;
    explicit AllocStreamScope(cudaStream_t s) : prev(g_alloc_stream) { g_alloc_stream = s; }
    ~AllocStreamScope() { g_alloc_stream = prev; }
};

// Injected faults (fds_fault_inject): true once, for the allocation or build
// that the armed fault names.
bool fds_fault_alloc_fires();
bool fds_fault_nan_fires();

// Device buffer owned by the handle (freed in the destructor).
template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaStream_t st = 0;   // stream the buffer was allocated on (and is freed on)
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n), st(o.st) { o.p = nullptr; o.n = 0; }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p; n = o.n; st = o.st;
            o.p = nullptr; o.n = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void release() {
        if (p) {
            if (st) cudaFreeAsync(p, st);
            else cudaFree(p);
        }
        p = nullptr;
        n = 0;
    }
    int alloc(size_t count) {
        release();
        if (count == 0) count = 1;
        st = g_alloc_stream;
        if (fds_fault_alloc_fires()) return FDS_ERR_OOM;
        cudaError_t e = st ? cudaMallocAsync((void **)&p, count * sizeof(T), st)
                           : cudaMalloc((void **)&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? FDS_ERR_OOM : FDS_ERR_CUDA;
        }
        n = count;
        return FDS_OK;
    }
    int upload(const std::vector<T> &h, cudaStream_t s) {
        int rc = alloc(h.size());
        if (rc != FDS_OK) return rc;
        if (!h.empty()) FDS_CUDA_TRY(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
        return FDS_OK;
    }
    size_t bytes() const { return n * sizeof(T); }
};

// One tree level: its cells, their active DOFs and (for compressed levels) the
// stored factors of Sec. 7.3 step 3(b).
// One launch of the tensor-core block products of the forward operator
// (fw_tc.cu): jobs y[ymap] (+)= op(A_e) x[xmap], op(A_e) m x k complex with
// k <= 128 (wider blocks are split into passes, one launch each).
struct OzJob {
    int64_t a_tile;      // first operator slice tile (16 KB each)
    int64_t x_tile;      // first vector slice group (sum of nkc over earlier jobs)
    int64_t x_row, y_row;   // row offsets into x and y
    int32_t xmap, ymap;     // offsets into the plan's map array (-1: rows contiguous)
    int32_t m, k;           // complex rows and columns of op(A_e)
    int32_t nmt, nkc;       // 128-real row tiles, 64-real K chunks
    int32_t rexp;           // first row exponent (nmt * 128 entries)
    int32_t flags;          // 1: y = product (y is not read)
};
struct OzPlan {
    int njobs = 0, ntiles = 0;   // ntiles: (job, row tile) pairs
    int64_t xgroups = 0;         // sum of nkc over the jobs
    double flops = 0;            // 8 m k per column, summed over the jobs
    DBuf<OzJob> jobs;
    DBuf<int2> tiles;            // (job, row tile)
    DBuf<int> maps;
    DBuf<unsigned char> aslices;
    DBuf<int> rowexp;
};

struct Level {
    int nb = 0;                  // cells
    // --- DOFs: per cell, comp-1 DOF nodes then comp-2 DOF nodes
    std::vector<int> n1, n2;
    std::vector<int64_t> doff;   // nb+1, prefix of n1+n2
    std::vector<int> dof_node;
    // union node list per cell (node, position in comp-1 list, in comp-2 list, group tag)
    std::vector<int64_t> uoff;   // nb+1
    std::vector<int> unode, upos1, upos2, utag;
    DBuf<int> d_unode, d_upos1, d_upos2, d_utag;
    DBuf<int64_t> d_uoff;
    // --- geometry of the cells (levels > l0 only)
    std::vector<double> cx, cy, R, Rp;
    std::vector<int> mprox;
    // --- compression
    std::vector<int> k1, k2;     // ranks
    std::vector<int64_t> permoff;   // 2 nb + 1 (index 2b + c)
    std::vector<int> perm;
    // --- factors (device), offsets in complex entries
    std::vector<int64_t> offA, offW, offAt, offV, offpiv;
    DBuf<cplx> LU, W, At, V, Ainv;   // LU: during the build only; Ainv = A_i^{-1} for the sweep
    DBuf<int> piv;
    DBuf<MatRef> rLU, rW, rAt, rV, rAinv;
    // FDS_VARIANT_MR2005: E_i = A_i^{-1} U_i A~_i (d x r), F_i = A~_i V_i A_i^{-1}
    // (r x d), G_i = A_i^{-1} - E_i V_i A_i^{-1} (d x d)
    DBuf<cplx> mrE, mrF, mrG;
    DBuf<MatRef> rmrE, rmrF, rmrG;
    DBuf<int64_t> d_offpiv;
    // --- placement of each cell's skeleton vector in its parent's DOF vector
    std::vector<int> par_pos1, par_pos2;   // start of comp-1 / comp-2 skeleton block in the parent
    DBuf<int> d_par_pos1, d_par_pos2, d_k1, d_k2;
    DBuf<int64_t> d_doff, d_roff;          // DOF / skeleton offsets (prefix of d and r)
    std::vector<int64_t> roff;
    int64_t D = 0, Rtot = 0;               // total DOFs / total skeleton DOFs of the level
    int dmax = 0, rmax = 0;
    double sum_d2 = 0, sum_rd = 0, sum_r2 = 0;   // algorithmic work sums for the sweep
    bool c64 = false;            // FDS_MIXED: merged and swept in complex64
    // --- interpolation blocks T^c (k_c x (n_c - k_c) per cell and component,
    //     offsets toff[2b + c]) and the cell-local permuted DOF order vmap
    //     (skeleton DOFs of each component first), for the structured V
    DBuf<cplx> T;
    DBuf<cplxf> Tf;
    DBuf<float4> Tp;
    DBuf<int64_t> d_toff;
    DBuf<int> d_vmap, d_n1, d_n2;
    int kmax = 0;                // largest k_c of the level
    double sum_tm = 0;           // sum over cells and components of k_c (n_c - k_c)
    // --- mixed precision: complex64 copies of the sweep factors
    DBuf<cplxf> Ainvf, Wf, Atf, Vf;
    DBuf<MatRefF> rAinvf, rWf, rAtf, rVf;
    // --- mixed precision with double-float levels: float-pair copies
    DBuf<float4> Ainvp, Wp, Atp;
    DBuf<MatRefP> rAinvp, rWp, rAtp;
    // --- FP64 compressed forward operator: leaf diagonal blocks (leaf level)
    //     and sibling-coupling blocks S (levels that are parents), both d x d;
    //     as float pairs (float4 per entry) when the residual runs double-float
    DBuf<cplx> Dfw, Sfw;
    DBuf<MatRef> rDfw, rSfw;
    DBuf<float4> Dp, Sp, Vp;
    DBuf<MatRefP> rDp, rSp, rVp;
    // --- the sibling coupling as its two nonzero blocks per parent cell:
    //     entry 2p = rows of child a x columns of child b, 2p + 1 the other;
    //     sperm: the parent's DOFs grouped by child (a's first)
    DBuf<cplx> Sc;
    DBuf<float4> Scp;
    DBuf<int64_t> d_scoff;
    DBuf<int> d_sperm, d_ra, d_rb;
    // --- fw_engine = FDS_FW_TENSOR (leaf level): bf16 slices of the diagonal
    //     blocks in pre-swizzled tensor-core tiles and their row exponents
    DBuf<unsigned char> oz_a;
    DBuf<int> oz_rowexp;
    // fw_engine = FDS_FW_TENSOR: plans of the level's forward-operator
    // products on the tensor cores (one entry per K pass): downward
    // interpolation (T^cH) and sibling blocks
    std::vector<OzPlan> oz_up, oz_down, oz_sib;
    std::vector<int64_t> toff_h;   // host copy of the T^c block offsets
    int srmax = 0;
    double sum_s2 = 0;            // sum over cells of 2 r_a r_b
};

// A stream created for (and destroyed after) one handle.
struct OwnedStream {
    cudaStream_t s = 0;
    ~OwnedStream() {
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    }
};

struct fds_handle {
    OwnedStream owned;      // first member: destroyed after every buffer below
    int N = 0;
    fds_physics ph{};
    PhysDev P{};
    double tol = 0;
    fds_options opt{};
    int L = 0, l0 = 0;
    cudaStream_t stream = 0;
    DBuf<double> d_xy;
    DBuf<int> d_leaf_gidx;        // leaf DOF q -> node + comp * N
    std::vector<double> xy;
    // ranges[l][i] = [lo, hi) node range of cell i at level l
    std::vector<std::vector<std::pair<int, int>>> ranges;
    std::vector<Level> lv;       // index = level (0..L); only l0..L populated
    // top system
    int64_t Dtop = 0;
    DBuf<cplx> Atop;
    DBuf<int> ptop;
    DBuf<MatRef> rtop;
    DBuf<cplx> Atop_inv;         // A_top^{-1} (the sweep's top solve is one GEMM)
    DBuf<MatRef> rtop_inv;
    DBuf<int64_t> d_ptop_off;
    DBuf<int> d_info;
    // mixed precision: off-diagonal top blocks (FP64 forward operator)
    DBuf<cplx> Atop_off;
    DBuf<MatRef> rtop_off;
    DBuf<float4> Atop_offp;
    DBuf<MatRefP> rtop_offp;
    // solve workspace (grown on demand)
    std::vector<DBuf<cplx>> wz, wf, wt, wy, wr;
    std::vector<DBuf<cplxf>> wzf, wff, wtf, wrf;
    DBuf<cplx> wtop, wytop, wX;
    DBuf<cplx> wtop2;                 // output of the top solve's GEMM
    DBuf<cplxf> wtopf;   // complex64 top vector (boundary of the mixed sweep)
    std::vector<DBuf<float4>> wzq, wfq, wtq, wrq;   // float-pair sweep vectors
    DBuf<float4> wtopq;
    DBuf<MatRefP> wrefsq;
    // forward-apply vectors as float pairs
    std::vector<DBuf<float4>> wzp, wtp, wyp;
    DBuf<float4> wtopp, wytopp, wXp;
    DBuf<MatRefP> wrefsp;
    DBuf<unsigned char> wvref;   // descriptors of the structured V applications
    DBuf<MatRef> wrefs;
    DBuf<MatRefF> wrefsf;
    DBuf<double> wnorm;
    DBuf<int> wundo;           // per-column flags of the refinement's take-back step
    DBuf<int> wcmap;           // refinement: right-hand side of each compact column
    DBuf<unsigned char> wperm; // refinement: staging of a column permutation
    bool oz_jobs = false;      // fw_engine = FDS_FW_TENSOR: the forward operator runs the levels' plans
    DBuf<unsigned char> oz_x;  // fw_engine = FDS_FW_TENSOR: bf16 slices of the vectors
    DBuf<int> oz_colexp;
    // use_graph: one CUDA graph of the sweep per column count, with the
    // workspace layout (hash of its buffer addresses) it was captured against
    struct SweepGraph {
        cudaGraphExec_t exec = nullptr;
        uint64_t ws_hash = 0;
    };
    std::vector<std::pair<int, SweepGraph>> sweep_graphs;
    ~fds_handle() {
        for (auto &g : sweep_graphs)
            if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
    }
    int64_t ws_cols = 0;
    double build_ms = 0, solve_ms = 0;
    int64_t factor_bytes = 0;
    // learned-rank ID: network parameters (device), counters, recorded training rows
    DBuf<float> d_mlp;
    int64_t id_sketched = 0, id_fallback = 0;
    std::vector<float> feat_rows, frac_rows;
    bool fp64_reached = false; // build: a complex128 level has been merged (all above are too)
    int ir_iters = 0;          // refinement sweeps of the last mixed solve
    double ir_residual = 0;    // max_c ||f_c - A x_c|| / ||f_c|| after the last mixed solve
};

// Per-cell descriptors of blocks stored back to back at base + off[b].
template <class C>
int make_refs_t(DBuf<MatRefT<C>> &dst, C *base, const std::vector<int64_t> &off, const std::vector<int> &rows,
                const std::vector<int> &cols, cudaStream_t s) {
    std::vector<MatRefT<C>> h(rows.size());
    for (size_t b = 0; b < rows.size(); ++b) {
        h[b].p = base + off[b];
        h[b].rows = rows[b];
        h[b].cols = cols[b];
        h[b].ld = rows[b] > 1 ? rows[b] : 1;
    }
    return dst.upload(h, s);
}

int fds_build_impl(fds_handle *h);
// FDS_VARIANT_MR2005: the Woodbury products E_i, F_i, G_i of a merged level
// (needs A_i^{-1}, W_i = A_i^{-1} U_i, A~_i and the dense V_i); dv, rv per cell.
int mr2005_level_factors(fds_handle *h, Level &C, const std::vector<int> &dv, const std::vector<int> &rv,
                         cudaStream_t s);
// FDS_MIXED: copy of a level's square blocks (LU buffer, before it is factored)
// into a forward-operator store.
int fds_keep_blocks(const Level &Lv, DBuf<cplx> &dst, DBuf<MatRef> &rdst, cudaStream_t s);
// FDS_MIXED: complex64 copies of the sweep factors below the top; releases
// the FP64 ones that the sweep no longer needs (the top LU stays FP64).
int fds_mixed_prepare(fds_handle *h);
int fds_solve_mixed_impl(fds_handle *h, cplx *d_rhs, int nrhs, cudaStream_t s);
int fds_solve_impl(fds_handle *h, cplx *d_rhs, int nrhs, cudaStream_t s);
int fds_rhs_impl(fds_handle *h, const int *d_kinds, const double *d_angles, int nrhs, cplx *d_f, cudaStream_t s);
