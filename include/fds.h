/*
 * fds.h — C ABI of the GB300 (sm_103a) fast direct solver for 2D time-harmonic
 * elastic wave scattering by a traction-free cavity, after arXiv 2411.18026.
 *
 * The solver factors the Galerkin P1 Burton–Miller system A x = f of Sec. 4
 * (A = D + I_0/2 + alpha N, eq. (Aijpq) and the blocks defined with it) with
 * the proxy-surface compression of Sec. 7 and the LU-based variant of the
 * Martinsson–Rokhlin solver of Sec. 6, then solves for any number of
 * right-hand sides.  Every step runs in this library's CUDA kernels on one GPU.
 *
 * Conventions shared by every entry point
 *   - Return value: FDS_OK (0) on success, a negative FDS_ERR_* code otherwise;
 *     fds_error_string() names it.  No C++ exception crosses the ABI.
 *   - Complex numbers are two adjacent doubles (re, im), i.e. C99
 *     double _Complex / cuDoubleComplex layout.
 *   - Geometry: a closed polygon with n nodes, coordinates interleaved
 *     (x0, y0, x1, y1, ...), nodes counter-clockwise around the cavity so the
 *     element normal (tangent rotated by +90 degrees) points into the cavity,
 *     the orientation Sec. 2 prescribes.  Element e joins node e to e+1 mod n.
 *   - Unknown layout (eq. (discre_x) applied to the whole vector): entry s is
 *     component 1 of the displacement at node s, entry n + s component 2.
 *     Multi-RHS arrays are column-major, 2n rows, one column per right-hand side.
 *   - Host pointers are read (or written) during the call only and stay owned
 *     by the caller.  Device pointers (d_ prefix) must be device-accessible
 *     memory of the current device; the call enqueues work on the given stream
 *     and returns without synchronising unless stated.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef FDS_H
#define FDS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDS_OK                 0
#define FDS_ERR_ARG           -1  /* invalid argument (null pointer, size, option) */
#define FDS_ERR_CUDA          -2  /* a CUDA runtime call failed */
#define FDS_ERR_OOM           -3  /* device allocation failed */
#define FDS_ERR_SINGULAR      -4  /* zero or non-finite pivot in a box LU, S_i or the top LU */
#define FDS_ERR_NOT_CONVERGED -5  /* iterative refinement did not reach its target */
#define FDS_ERR_TIMEOUT       -6  /* a device-side wait exceeded its iteration budget */
#define FDS_ERR_STATE         -7  /* handle not in a state that allows the call */

#define FDS_FP64  0               /* all arithmetic in FP64 / complex128 */
#define FDS_MIXED 1               /* FP64 build; complex64 sweep refined against the FP64
                                     compressed forward operator */
#define FDS_APPLY_FF   0
#define FDS_APPLY_FP64 1

/* Skeleton selection (Sec. 7.2): adaptive CPQR on the stacked proxy matrix,
 * or (extension, not in the paper) a rank predicted by the learned network
 * from geometry features, a sparse-sign sketch of the proxy matrix with
 * (predicted rank + sketch_extra) rows, CPQR of the sketch, and a check of
 * the ID residual on the whole proxy matrix against the adaptive CPQR's own
 * bound; cells that fail the check fall back to the adaptive CPQR. */
/* Engine of the complex64 products (sweep levels below the double-float ones,
 * and the merges with merge_c64 = 1): plain FP32 FMA, or the tensor cores
 * (tcgen05, each fp32 operand split into three bf16 pieces, six products,
 * fp32 accumulation in tensor memory). */
#define FDS_C64_SIMT   0
#define FDS_C64_TENSOR 1
/* Engine of the refinement's forward operator (FDS_MIXED with
 * FDS_APPLY_FF): double-float products on the FP32 pipe, or the tensor cores
 * for the leaf diagonal blocks (leaves of at most 64 nodes; larger ones stay
 * double-float), the sibling blocks and the interpolation blocks, with the
 * FP64 blocks and the vectors cut into six bf16 slices each (per-row /
 * per-column powers of two), the 21 slice products with i + j <= 5
 * accumulated in fp32 tensor memory (exact for the leading groups) and
 * summed in float pairs: about 2^-40 of |A| |x|, against 2^-44 for the
 * double-float products. */
#define FDS_FW_FF     0
#define FDS_FW_TENSOR 1

/* Elimination variant (Sec. 6): the paper's LU-based recursion (default), or
 * the Sherman–Morrison–Woodbury form of the original Martinsson–Rokhlin
 * method it is compared with (Sec. 6 introduction), which additionally forms
 * E_i = A_i^{-1} U_i A~_i, F_i = A~_i V_i A_i^{-1} and
 * G_i = A_i^{-1} - A_i^{-1} U_i A~_i V_i A_i^{-1} per cell and solves by
 * f~_i = F_i f_i upward and x_i = G_i f_i + E_i y_i downward; FDS_FP64 only. */
#define FDS_VARIANT_LU     0
#define FDS_VARIANT_MR2005 1

#define FDS_RANK_ADAPTIVE 0
#define FDS_RANK_LEARNED  1
/* Learned-rank network: 16 -> 64 -> 64 -> 1, tanh, FP32.  Parameter vector:
 * W1 [64x16] row-major, b1 [64], W2 [64x64], b2 [64], w3 [64], b3 (trained),
 * then input normalisation mu [16], sd [16]. */
#define FDS_MLP_NIN    16
#define FDS_MLP_NTRAIN 5313
#define FDS_MLP_NPARAM 5345

typedef struct fds_handle fds_handle;   /* opaque; owns all device memory of one factorisation */

/* Material and frequency (Sec. 2): Lame constants lambda, mu, density rho,
 * angular frequency omega.  Burton–Miller coupling alpha (eq. (bie)); when
 * alpha_set == 0 the library uses alpha = i / (mu k_T), k_T = omega sqrt(rho/mu). */
typedef struct {
    double lambda, mu, rho, omega;
    double alpha_re, alpha_im;
    int32_t alpha_set;
} fds_physics;

typedef struct {
    int32_t n_nodes;       /* number of polygon nodes = number of elements, >= 8 */
    const double *xy;      /* host, 2*n_nodes doubles, see conventions */
    double rho;            /* density; <= 0 means 1 */
} fds_geometry;

typedef struct {
    int32_t leaf_size;     /* maximum nodes per leaf cell n (Sec. 5.1); default 64 */
    double proxy_ratio;    /* proxy circle radius / cell radius (Sec. 7.1); default 1.5 */
    int32_t proxy_points;  /* minimum proxy polygon vertices m'; default 64; the library
                              uses max(proxy_points, ceil(2 k_T R_proxy + 30)) */
    int32_t top_level;     /* level l0 of the dense top solve (Sec. 7.3); default 1; clamped to
                              the depth L.  Negative: l0 = max(L + top_level, 0), so -1 is the
                              single-level variant of Sec. 8.1 (Table tab:error_single: only
                              the leaf cells are compressed and their skeleton system is
                              factored densely; O(N^3) in the top LU) */
    int32_t precision;     /* FDS_FP64 (default) or FDS_MIXED */
    double alpha_re, alpha_im;
    int32_t alpha_set;     /* 0: alpha = i/(mu k_T) */
    uint64_t cuda_stream;  /* cudaStream_t for the build; 0 = legacy default stream */
    double ir_tol;         /* FDS_MIXED: stop refining when max over right-hand sides of
                              ||f - A x|| / ||f|| <= ir_tol (A = compressed operator); default 1e-9 */
    int32_t ir_max_iter;   /* FDS_MIXED: maximum refinement sweeps after the first; default 10;
                              0 gives the plain complex64 sweep */
    int32_t ir_apply;      /* FDS_MIXED: arithmetic of the forward operator in the residual:
                              FDS_APPLY_FF (default) double-float products and sums on the
                              FP32 pipe (about 44 significant bits), FDS_APPLY_FP64 FP64 */
    int32_t sweep_fp64_levels; /* FDS_MIXED: tree levels below the top whose sweep factors stay
                              complex128 (the rest are complex64; the rounding error of the
                              complex64 sweep comes mostly from the upper levels); -1 (default):
                              the levels with at most 1/8 of the leaf level's DOFs */
    int32_t sweep_ff;      /* FDS_MIXED: the levels above the complex64 ones sweep in 0 complex128,
                              1 (default) double-float arithmetic on the FP32 pipe (float pairs,
                              ~44 bits); 2: every level in double-float (no complex64 level) */
    int32_t merge_c64;     /* FDS_MIXED: 1 merges the complex64 levels in complex64 too (faster
                              build; their rounding then also enters the upper levels'
                              factors, so refinement may need more sweeps); default 0 */
    int32_t rank_mode;     /* FDS_RANK_ADAPTIVE (default) or FDS_RANK_LEARNED */
    const float *mlp_params; /* FDS_RANK_LEARNED: host, FDS_MLP_NPARAM floats, copied at the call */
    int32_t sketch_extra;  /* FDS_RANK_LEARNED: sketch rows beyond the predicted rank; default 12 */
    int32_t record_features; /* 1: keep the features and adaptive ranks of every (cell, component)
                              for fds_features_get (training data) */
    int32_t c64_engine;    /* FDS_MIXED: FDS_C64_SIMT (default) or FDS_C64_TENSOR; the tensor
                              cores' fp32 accumulation is less accurate than fp32 FMA, which
                              can cost the refinement an extra sweep */
    double tol_decay;      /* ID tolerance per level: tol at the leaf level L and
                              tol * tol_decay^(L - l) at level l (0 < tol_decay <= 1),
                              but not below min(tol, 1e-15).  Default 0.5.  1 gives the
                              paper's single tolerance at every level, whose error grows
                              with the depth (Sec. 8.1, Table tab:error); halving the
                              tolerance per level up keeps the error near tol (measured:
                              error / tol <= 2.1 at 2^12-2^13 nodes, against 4-28 with 1) */
    int32_t variant;       /* FDS_VARIANT_LU (default) or FDS_VARIANT_MR2005 (FDS_FP64 only) */
    int32_t use_graph;     /* 1: each solve sweep (all levels up, top, all levels down, for one
                              column chunk) replays a CUDA graph captured on the first sweep of
                              that column count, instead of launching its kernels one by one;
                              needs a non-default stream (handles built by fds_build_batch
                              have one); default 0 */
    int32_t fw_engine;     /* FDS_MIXED: FDS_FW_FF (default) or FDS_FW_TENSOR for the leaf,
                              sibling and interpolation blocks of the refinement's forward
                              operator */
    int32_t merge_c64_levels; /* with merge_c64 = 1: only the lowest merge_c64_levels of the
                              complex64 levels are merged in complex64, the others in FP64;
                              0 (default): all of them */
} fds_options;

/* Statistics of a built handle. */
typedef struct {
    int32_t n_nodes, levels, top_level, top_size;
    int64_t skeleton_dofs[32];   /* sum of ranks k^1 + k^2 over the cells of level l */
    int32_t max_rank[32];        /* largest k^1 + k^2 of a cell at level l */
    double build_ms;             /* device time of the last fds_build (CUDA events) */
    double solve_ms;             /* device time of the last fds_solve*/
    int64_t factor_bytes;        /* device bytes held by the factors */
    int32_t ir_iters;            /* FDS_MIXED: refinement sweeps of the last solve */
    double ir_residual;          /* FDS_MIXED: final max relative residual of the last solve */
    int64_t id_sketched;         /* FDS_RANK_LEARNED: (cell, component) IDs accepted from the sketch */
    int64_t id_fallback;         /* FDS_RANK_LEARNED: IDs redone by the adaptive CPQR */
    int64_t features_recorded;   /* rows available to fds_features_get */
} fds_stats;

/* Fill *o with the defaults listed above. */
void fds_default_options(fds_options *o);

/*
 * Build: geometry + tree (Sec. 5.1), then for l = L .. l0+1 the proxy
 * compression of Sec. 7 (kernel evaluation, interpolative decomposition by
 * column-pivoted QR with relative tolerance tol), the upward elimination of
 * Sec. 6.2 (LU of A_i, A_i^{-1} U_i, A~_i = (V_i A_i^{-1} U_i)^{-1}) and the
 * parent rearrangement of eq. (A_rearrangement); finally the dense LU of the
 * level-l0 system (Sec. 6.3).  omega > 0, lambda > -mu (so lambda+2mu > 0),
 * mu > 0, 0 <= tol < 1.  On success *out receives a new handle.
 */
int fds_build(const fds_geometry *g, double omega, double lambda, double mu, double tol,
              fds_handle **out);
int fds_build_ex(const fds_geometry *g, double omega, double lambda, double mu, double tol,
                 const fds_options *opt, fds_handle **out);

/*
 * Galerkin load vectors f^s_i = int psi^s (u^I_i + alpha T^{n_x}_ij u^I_j) ds
 * (Sec. 4) for plane waves of direction d = (cos a, sin a): kinds[r] = 0 is a
 * P wave u^I = d exp(i k_L d.x), 1 an SV wave u^I = d_perp exp(i k_T d.x),
 * d_perp = (-d_2, d_1).  f_out: host, 2n x nrhs complex, column-major.
 */
int fds_rhs_plane_wave(fds_handle *h, const int32_t *kinds, const double *angles, int32_t nrhs,
                       double *f_out);
/* Same on the device: d_kinds, d_angles, d_f device arrays; enqueued on stream. */
int fds_rhs_plane_wave_device(fds_handle *h, const int32_t *d_kinds, const double *d_angles,
                              int32_t nrhs, double *d_f, uint64_t stream);

/*
 * Solve A x = f for nrhs right-hand sides (Sec. 6.2-6.3): upward pass
 * z_i = A_i^{-1} f_i, f~_i = A~_i V_i z_i (eq. (linear_last)), top solve,
 * downward pass x_i = z_i - W_i (f~_i - A~_i y_i), W_i = A_i^{-1} U_i
 * (eq. (down_comv)).
 * FDS_MIXED: the sweep runs on complex64 copies of the factors (the top
 * solve stays FP64) and is
 * repeated on the residual r = f - A x, where A is the compressed operator
 * the factorisation inverts (leaf diagonal blocks, interpolation matrices,
 * original entries between sibling skeletons and between top cells), applied
 * in FP64; it stops when max_c ||r_c|| / ||f_c|| <= ir_tol, after ir_max_iter
 * extra sweeps, or when the residual stops halving.  If the target was not
 * met the solution reached is still written and FDS_ERR_NOT_CONVERGED is
 * returned; fds_stats_get reports the sweeps and the final residual.
 * fds_solve: host rhs (2n x nrhs complex, column-major), copied to the device,
 * solved, copied back in place; synchronous.  fds_solve_device: d_rhs on the
 * device, overwritten in place, enqueued on stream (FDS_MIXED synchronises
 * the stream once per refinement sweep to read the residual norms).
 */
int fds_solve(fds_handle *h, double *rhs, int32_t nrhs);
int fds_solve_device(fds_handle *h, double *d_rhs, int32_t nrhs, uint64_t stream);

int fds_stats_get(const fds_handle *h, fds_stats *s);
/* Per-cell skeleton ranks of level l (L >= l > l0): k[2*i + c] for cell i,
 * component c.  cap = capacity of k in int32 entries; returns the count or an
 * error. */
int fds_level_ranks(const fds_handle *h, int32_t level, int32_t *k, int32_t cap);
void fds_destroy(fds_handle *h);   /* NULL-safe; frees every device buffer of h */
const char *fds_error_string(int code);
/* The CUDA error name, message and source location behind the last
 * FDS_ERR_CUDA / FDS_ERR_OOM returned to the calling thread ("" if none);
 * valid until the thread's next failing call. */
const char *fds_last_error_detail(void);

/*
 * Per-phase device timing: when enabled, the library brackets its kernel
 * launches with CUDA events on the launch stream and accumulates, per phase
 * name, the launch count, the summed device time and the algorithmic work
 * (flops, bytes) the phase performs, and for quadrature phases the number of
 * quadrature point evaluations (units).  Off by default; process-wide.
 * fds_timing_report writes lines "name launches total_ms flops bytes units" into
 * buf (at most cap bytes, NUL-terminated) and returns the length it needs.
 * Reporting synchronises on the recorded events.
 */
void fds_timing_enable(int32_t on);
void fds_timing_reset(void);
int fds_timing_report(char *buf, int32_t cap);
/* Number of kernels this library has launched since it was loaded. */
int64_t fds_launch_count(void);
/*
 * Measured arithmetic peak of the current device (a measurement service, not
 * a step of the paper's method): kind 0 FP64, 1 FP32.  A register-resident
 * loop of independent fused multiply-adds on 8 blocks of 256 threads per SM,
 * calibrated to ~60 ms per launch, best of three launches timed with CUDA
 * events on the legacy default stream; *tflops receives 2 x FMAs / second
 * / 1e12 at whatever clock the GPU ran.  Allocates 8 bytes of device memory
 * for the duration of the call; synchronous.
 */
int fds_alu_peak(int32_t kind, double *tflops);

/*
 * Tile autotuner of the batched register-tiled GEMMs (the complex64,
 * complex128 and double-float products of the merges, the solve sweep and
 * the forward operator; an extension, not in the paper).  When enabled, the
 * first launch of each shape class (arithmetic, op(A), row count rounded up
 * to 16, column count and batch size rounded up to powers of two, with or
 * without row maps) whose result does not read C (beta = 0) times every
 * candidate tile shape (row groups x columns per thread) on its stream with
 * CUDA events, best of two, synchronising the stream, and records the
 * fastest in a process-wide table that later launches of the class use;
 * classes not yet tuned, and launches during stream capture, use the fixed
 * rule (tile height that pads the rows least).  Every candidate accumulates
 * over K in the same order, so results do not depend on the shape chosen.
 * fds_autotune_report writes one line per class: "arith opA rows cols batch
 * mapped MI TJ best_us rule_us" into buf (cap bytes, NUL-terminated) and
 * returns the length it needs.  Process-wide; off by default.
 */
void fds_autotune_enable(int32_t on);
void fds_autotune_reset(void);
int fds_autotune_report(char *buf, int32_t cap);

/*
 * Fault injection for tests of the failure paths (an extension, not in the
 * paper).  Every fault is made on the host or by withholding work, never by
 * a bad access: the device context stays usable afterwards.  An armed fault
 * fires once and then disarms itself.
 *   FDS_FAULT_NONE         disarm every fault (arg ignored).
 *   FDS_FAULT_ALLOC        the arg-th device allocation of the library from
 *                          now on (arg >= 1) fails as if the device were out
 *                          of memory: the call returns FDS_ERR_OOM after
 *                          freeing what it had allocated.
 *   FDS_FAULT_NAN_BLOCK    the next build writes a NaN into the first entry
 *                          of the first leaf's diagonal block after the
 *                          kernel evaluation: the block LU meets a
 *                          non-finite pivot and the build returns
 *                          FDS_ERR_SINGULAR.
 *   FDS_FAULT_TC_STALL_FW  in the next launch of the tensor-core leaf-block
 *                          product (fw_engine = FDS_FW_TENSOR,
 *                          fds_zgemm_blocks_tc), the first CTA's producer
 *                          issues no copies: its MMA thread's bounded wait
 *                          (about 2 s) runs out, the kernel records a status,
 *                          frees its tensor memory and returns; the call
 *                          returns FDS_ERR_TIMEOUT.
 *   FDS_FAULT_TC_STALL_C64 the same for the complex64 tensor-core GEMM
 *                          (FDS_C64_TENSOR, fds_cgemm_c64_batched): the first
 *                          CTA issues no MMAs, so its completion waits run out.
 * Returns FDS_OK, FDS_ERR_ARG (unknown kind, arg < 1 for FDS_FAULT_ALLOC) or
 * FDS_ERR_CUDA (the device flag of a stall could not be set).  Process-wide;
 * not meant to be armed while another thread builds or solves.  The
 * environment variable FDS_FAULT ("alloc:N", "nan", "stall_fw" or
 * "stall_c64") arms the same fault once per process, at the first build.
 */
/*
 * Bounds-checked build: a library compiled with -DFDS_CHECKS
 * (paper_2411_18026_gb300/libfds_checked.so, build(checked=True)) checks
 * every index-mapped gather and scatter (row maps of the batched GEMMs, the
 * skeleton and child-to-parent placements, the leaf-order permutation)
 * against the extent of the buffer it addresses, skips an access out of
 * range and counts it.  fds_bounds_violations synchronises the device and
 * writes the count since the previous call (then resets it) to *count;
 * FDS_ERR_STATE in a library built without the checks.
 */
int fds_bounds_violations(int64_t *count);

#define FDS_FAULT_NONE 0
#define FDS_FAULT_ALLOC 1
#define FDS_FAULT_NAN_BLOCK 2
#define FDS_FAULT_TC_STALL_FW 3
#define FDS_FAULT_TC_STALL_C64 4
int fds_fault_inject(int32_t kind, int64_t arg);

/* ------------------------------------------------------------------------
 * Stage entry points: each runs one step of the hot path on caller-provided
 * device buffers, so that it can be checked on its own.  All enqueue on
 * `stream` and do not synchronise.
 * ------------------------------------------------------------------------ */

/*
 * Kernel evaluation (Sec. 4, eq. (Aijpq); singular pairs by the regularised
 * Galerkin forms): block A(rows, cols) of the boundary matrix
 * D + I_0/2 + alpha N between test hats d_rows[0..nr) and trial hats
 * d_cols[0..nc) on the polygon d_xy (n nodes).  d_out: complex, column-major,
 * (2 nr) x (2 nc), leading dimension 2 nr; row r + i nr is component i+1 of
 * hat d_rows[r], column c + j nc component j+1 of hat d_cols[c].
 */
int fds_eval_entries(const fds_physics *ph, const double *d_xy, int32_t n, const int32_t *d_rows,
                     int32_t nr, const int32_t *d_cols, int32_t nc, double *d_out, uint64_t stream);

/*
 * Proxy interaction entries (Sec. 7, eq. (mv) and the matrix M^U): D + alpha N
 * between test hats d_rows on closed polygon X (nx nodes) and trial hats
 * d_cols on closed polygon Y (ny nodes), fixed q x q Gauss rule per element
 * pair (1 <= q <= 8), no mass term.  Output layout as fds_eval_entries.
 */
int fds_eval_cross(const fds_physics *ph, const double *d_X, int32_t nx, const int32_t *d_rows,
                   int32_t nr, const double *d_Y, int32_t ny, const int32_t *d_cols, int32_t nc,
                   int32_t q, double *d_out, uint64_t stream);

/*
 * Interpolative decomposition (Sec. 7.1) of a batch of complex matrices by
 * Householder QR with column pivoting (largest remaining column 2-norm, ties to
 * the lowest index), truncated at the first pivot with |R_jj| <= tol |R_11|.
 * Matrix b: m[b] x n[b], column-major at d_Y + 2*off[b] doubles, leading
 * dimension m[b]; overwritten by the QR factors.  Outputs: d_rank[b] = k,
 * d_perm + poff[b]: the n[b] column indices in pivot order,
 * d_T + 2*toff[b] doubles: T = R_1^{-1} R_2, k x (n-k) column-major (leading
 * dimension k), so that Y[:, perm[k:]] ~= Y[:, perm[:k]] T.  The T slot of
 * matrix b must hold k (n-k) <= n[b]^2/4 + 1 complex entries.
 */
int fds_id_batched(int32_t batch, const int32_t *d_m, const int32_t *d_n, const int64_t *d_off,
                   double *d_Y, double tol, int32_t *d_rank, int32_t *d_perm,
                   const int64_t *d_poff, double *d_T, const int64_t *d_toff, uint64_t stream);

/*
 * Batched LU with partial pivoting of square complex matrices (the box LU of
 * Sec. 7.3 step 3(b) and the top LU of step 4): matrix b is d[b] x d[b],
 * column-major at d_A + 2*off[b] doubles (leading dimension d[b]), overwritten
 * by L (unit, below the diagonal) and U; d_piv + poff[b] receives the pivot row
 * of each step.  d_info[b] = 0, or j+1 if the j-th pivot is zero or not finite.
 */
int fds_lu_batched(int32_t batch, const int32_t *d_d, const int64_t *d_off, double *d_A,
                   int32_t *d_piv, const int64_t *d_poff, int32_t *d_info, uint64_t stream);

/*
 * fds_lu_batched_noalloc: the batched LU above without any allocation, for
 * callers that cannot allocate device memory at the point of the call — for
 * example code running inside another allocator's callback, a process whose
 * device memory is reserved up front by a caching allocator so that a fresh
 * cudaMalloc may fail, or a latency-critical loop that must not pay for the
 * implicit synchronisation of cudaMalloc/cudaFree.  The paper has no
 * counterpart; this is a service of the library.
 * Same arguments, layout and results as fds_lu_batched.  The per-matrix
 * descriptors live in a static device array of FDS_LU_NOALLOC_MAX_BATCH
 * (16384) entries (384 KiB, held by every GPU that loads the library until
 * the process exits); batch > 16384 returns FDS_ERR_ARG.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * The address is kept per device ordinal for the life of the process: after
 * cudaDeviceReset() of a device the kept address is stale, so a process that
 * resets a device must not call this entry point on it again.
 * Every call shares the array, which keeps the last call's descriptors:
 * calls that overlap on the GPU (different streams, or different host
 * threads on the same device) race and must be serialised by the caller.
 * No cudaMalloc, cudaFree or other allocating call is made.
 */
int fds_lu_batched_noalloc(int32_t batch, const int32_t *d_d, const int64_t *d_off, double *d_A,
                           int32_t *d_piv, const int64_t *d_poff, int32_t *d_info, uint64_t stream);

/*
 * Displacement off the boundary (Sec. 3, eq. (integ_rep)), for the
 * traction-free cavity of handle h:
 *   u_i(x) = u^I_i(x) - int_Gamma T^{n_y}_{jk} G_ik(x - y) u_j(y) ds(y),
 * with u the boundary solution (P1 nodal values) and u^I the plane wave it
 * was solved for.  d_u: device, 2n x nrhs complex128, column-major in the
 * unknown layout above (as left by fds_solve_device); kinds/angles: host,
 * nrhs entries as given to fds_rhs_plane_wave (0 = P, 1 = SV); d_pts:
 * device, npts points (x, y interleaved) off the boundary (the 8-point rule
 * per element is accurate at distances of a few element lengths and more);
 * d_out: device, 2 npts x nrhs complex128, column j = component 1 at the
 * points, then component 2.  Direct summation over the elements
 * (O(n npts nrhs)); synchronises the stream.
 */
int fds_field(fds_handle *h, const double *d_u, int32_t nrhs, const int32_t *kinds, const double *angles,
              const double *d_pts, int32_t npts, double *d_out, uint64_t stream);
/*
 * The same field with the tree's proxy compression (Sec. 3 eq. (integ_rep)
 * evaluated through the skeletons of Sec. 7): a cell's boundary sources seen
 * from a point outside its proxy circle are replaced by its skeleton hats
 * with coefficients u~ = V u (recursively u~_parent = V_parent applied to the
 * children's u~); each point sums the skeletons of the largest cells (levels
 * l0+1 .. L) whose proxy circle it lies outside, and the hats of the leaf
 * cells whose proxy circle holds it directly.  Work per point
 * O(skeleton DOFs of those cells) instead of O(n).  Accuracy follows the ID
 * tolerance of the build.  Same arguments and layout as fds_field; the
 * points are read back to the host to choose each point's cells;
 * synchronises the stream.  FDS_ERR_STATE if the handle has no interpolation
 * blocks.
 */
int fds_field_compressed(fds_handle *h, const double *d_u, int32_t nrhs, const int32_t *kinds,
                         const double *angles, const double *d_pts, int32_t npts, double *d_out, uint64_t stream);

/*
 * Batched complex64 GEMM of the mixed-precision levels (Sec. 7.3 products in
 * complex64; stage entry for tests and benchmarks):
 *   C_b = alpha op(A_b) B_b + beta C_b,   b = 0 .. batch-1,
 * op = identity (opA 0) or conjugate transpose (opA 2); op(A_b) is m[b] x k[b],
 * B_b k[b] x n[b], C_b m[b] x n[b].  All column-major complex64 (re, im float
 * pairs) with leading dimension = rows, at d_A + 2*aoff[b], d_B + 2*boff[b],
 * d_C + 2*coff[b] floats (A_b stored k[b] x m[b] for opA 2).  alpha, beta real.
 * engine: FDS_C64_TENSOR (tcgen05, bf16 x 3 pieces) or FDS_C64_SIMT.  d_m, d_n, d_k,
 * d_*off are host arrays of batch entries; the call allocates (and frees,
 * after synchronising the stream) the device descriptors.  batch <= 65535.
 * FDS_ERR_TIMEOUT if a tensor-core wait gave up (the stream is synchronised).
 */
int fds_cgemm_c64_batched(int32_t batch, const int32_t *m, const int32_t *n, const int32_t *k,
                          const int64_t *aoff, const int64_t *boff, const int64_t *coff, const float *d_A,
                          const float *d_B, float *d_C, int32_t opA, float alpha, float beta, int32_t engine,
                          uint64_t stream);

/*
 * The tensor-core product of the forward operator's leaf blocks (stage entry
 * for tests and benchmarks; fw_engine = FDS_FW_TENSOR): Y_b += A_b X_b for
 * b < batch, A_b d[b] x d[b] complex128 (1 <= d[b] <= 128) stored column-major
 * back to back at d_A, X and Y the row blocks of one (sum d) x nc complex128
 * matrix (column-major, leading dimension sum d), block b at rows
 * sum_{c<b} d[c].  Operands are cut into six bf16 slices with per-row /
 * per-column powers of two and the 21 slice products with i + j <= 5 are
 * accumulated on the tensor cores (the vectors pass through float pairs, as
 * in the refinement).  d: host array.  Allocates its temporaries; synchronises
 * the stream; FDS_ERR_TIMEOUT if a tensor-core pipeline wait gave up.
 */
int fds_zgemm_blocks_tc(int32_t batch, const int32_t *d, const double *d_A, const double *d_X, double *d_Y,
                        int32_t nc, uint64_t stream);

/*
 * General block products of the forward operator on the tensor cores (stage
 * entry; the sibling and interpolation blocks with fw_engine =
 * FDS_FW_TENSOR use the same kernels): for each job e < njobs,
 *   Y[y_row[e] + ymap_e[i], :] (+)= sum_l op(A_e)[i][l] X[x_row[e] + xmap_e[l], :]
 * for i < m[e], l < k[e], where op(A_e) = A_e (op[e] = 0, stored m x k) or
 * A_e^H (op[e] = 1, stored k x m), the stored block column-major at
 * d_A + 2 a_off[e] doubles with leading dimension lda[e] (complex128).
 * xmap_e = maps + xmap_off[e] (k[e] entries) and ymap_e = maps + ymap_off[e]
 * (m[e] entries); an offset of -1 means rows taken in order (map = identity).
 * set[e] != 0: Y = product, else Y += product.  Jobs must write disjoint rows
 * of Y.  X (ldx) and Y (ldy) are complex128, column-major, nc columns, on the
 * device; all other arrays are host arrays.  Same slicing, accuracy and
 * float-pair vectors as fds_zgemm_blocks_tc; op(A_e) wider than 128 complex
 * columns runs as several passes.  Allocates its temporaries; synchronises
 * the stream; FDS_ERR_TIMEOUT if a tensor-core pipeline wait gave up.
 */
int fds_zgemm_jobs_tc(int32_t njobs, const int32_t *m, const int32_t *k, const int32_t *op, const int64_t *a_off,
                      const int32_t *lda, const int64_t *x_row, const int64_t *xmap_off, const int64_t *y_row,
                      const int64_t *ymap_off, const int32_t *set, const int32_t *maps, const double *d_A,
                      const double *d_X, int64_t ldx, double *d_Y, int64_t ldy, int32_t nc, uint64_t stream);

/*
 * Training data of the learned-rank network (extension): the 16 features of
 * each (cell, component) of levels L..l0+1 and the fraction k / n that the
 * adaptive ID kept there, recorded by a build with record_features = 1.
 * feat: host, cap x 16 floats; frac: host, cap floats.  Returns the number of
 * rows written (min(cap, recorded)) or an error.  Features, in order:
 * height above the leaves, log2 n, component, k_T 2R, k_L 2R, arc / 2R,
 * chord / arc, mean / max / RMS |turning angle|, total turning, sqrt of the
 * covariance eigenvalue ratio of the cell's vertices, near-field DOFs / d,
 * log10 tol, n / cell nodes, k_T arc / 2 pi.
 */
int fds_features_get(const fds_handle *h, float *feat, float *frac, int32_t cap);

/*
 * Learned-rank network kernels (device pointers, FP32, enqueued on stream).
 * fds_mlp_forward: y[b] = network(X[b, :]) for b < n.
 * fds_mlp_loss_grad: L = (1/n) sum_b (y_b - t_b)^2 and dL/dtheta
 *   (FDS_MLP_NTRAIN floats) over samples 0..n-1; deterministic.
 * fds_mlp_adam: one Adam step (Kingma & Ba, Algorithm 1) of the trained
 *   parameters with moment buffers m, v (FDS_MLP_NTRAIN floats each, zero at
 *   step 1); step counts from 1.
 * fds_mlp_train: Adam (0.9, 0.999, 1e-8) over the minibatches
 *   order[s*batch .. (s+1)*batch) for s < n_order / batch, moments starting
 *   at zero; losses (nullable) receives the loss of each step.
 */
int fds_mlp_forward(const float *d_params, const float *d_X, int32_t n, float *d_y, uint64_t stream);
int fds_mlp_loss_grad(const float *d_params, const float *d_X, const float *d_t, int32_t n, float *d_grad,
                      float *d_loss, uint64_t stream);
int fds_mlp_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, int32_t step, float lr,
                 float beta1, float beta2, float eps, uint64_t stream);
int fds_mlp_train(float *d_params, const float *d_X, const float *d_t, int32_t n, const int32_t *d_order,
                  int32_t n_order, int32_t batch, float lr, float *d_losses, uint64_t stream);

/*
 * Batched cavities (extension: many independent scatterers in one call).
 * fds_build_batch: count cavities (geometry g[i], angular frequency omega[i];
 * lambda, mu, tol and options shared, options.cuda_stream ignored) are built
 * concurrently by n_streams (1..64) host threads, each cavity on a stream
 * created for and owned by its handle (largest cavities first).  out[i]
 * receives cavity i's handle (release each with fds_destroy).  On any error
 * every handle of the batch is destroyed, out[] is cleared, and the first
 * error in cavity order is returned.
 * fds_solve_batch: solves d_rhs[i] (device, 2 n_i x nrhs[i], in place) with
 * handle h[i] on the handle's stream, n_streams threads; returns after all
 * solves have finished.
 * fds_handle_stream: the stream a handle runs on (its own for batched
 * handles), for enqueueing right-hand-side assembly on it.
 */
int fds_build_batch(int32_t count, const fds_geometry *g, const double *omega, double lambda, double mu,
                    double tol, const fds_options *opt, int32_t n_streams, fds_handle **out);
int fds_solve_batch(int32_t count, fds_handle *const *h, double *const *d_rhs, const int32_t *nrhs,
                    int32_t n_streams);
uint64_t fds_handle_stream(const fds_handle *h);

/*
 * Solve of many cavities with one launch per tree level and phase across all
 * of them (Sec. 7.3's sweep, whose cells of one level are independent, over
 * the cells of every cavity at once): for handles h[0..count) built with
 * precision FDS_FP64 and the LU variant, each with at least one level below
 * its top, the upward sweep runs aligned from the leaves (step j: level
 * L_i - j of every cavity that has it), the top solves as one batched GEMM,
 * the downward sweep aligned from the top; each phase of a step (Z =
 * A^{-1} R, the two parts of V, A~ U, the parent placement; downward the
 * gathers and the two updates) is one launch over the cells of all
 * participating cavities.  d_rhs[i]: device, 2 n_i x nrhs[i] complex128,
 * solved in place in chunks of 256 columns.  use_graph != 0 captures the
 * sweep of a chunk shape into a CUDA graph on its first chunk and replays
 * it for the later chunks of that shape (needs a non-default stream).
 * Waits for each handle's stream, runs on `stream`, synchronises it at the
 * end.  Results equal fds_solve's on each handle (same kernels, same
 * summation order).  FDS_ERR_ARG for a handle of another precision or
 * variant, or with a single cell.
 */
int fds_solve_batch_levels(int32_t count, fds_handle *const *h, double *const *d_rhs, const int32_t *nrhs,
                           int32_t use_graph, uint64_t stream);

#ifdef __cplusplus
}
#endif

#endif /* FDS_H */
