"""Benchmark of the GB300 fast direct solver.

One step = the whole hot path for one cavity: factorisation (cell circles,
near field, Galerkin kernel evaluation of leaf blocks and proxy/near rows,
CPQR interpolative decomposition, LU-based merges, top LU), the Galerkin load
vectors of all incident waves, and the multi-RHS solve sweep.

Default workload (the configuration the metric is quoted on): star cavity
r(t) = 1 + 0.2 cos 5t with 2^19 nodes (2^20 complex unknowns), lambda = 2,
mu = 1, rho = 1, k_T a = 20, leaf 64, l0 = 1, ID tolerance 1e-9 at the leaves
and halved per level up, 1000 right-hand sides (plane P and SV waves at 500
angles), learned rank (the trained network sizes a sketched ID, adaptive
CPQR as fallback), mixed precision (complex64 merges with Newton-refined
inverses and complex64 sweep of the lower tree levels, double-float sweep of
the upper ones, refined column by column against the FP64 compressed
operator, whose block products run on the tensor cores, to
||f - A x|| / ||f|| <= 1e-8).  After the timed
steps one plain-FP64 step (adaptive CPQR, FP64 merges and sweep) runs on the
same inputs: its build and solve times and the relative error between the
two solutions are reported beside the headline.  The working set (factors, vectors) is far larger than L2, so no
explicit flush is needed between steps.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank solves its own (rotated) copy of the cavity; there is
no collective in the data path, only a MAX reduction of the timings.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "build s + per-RHS µs at N=2^20, mixed/learned vs plain FP64, rel err ≤1e-6"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--nodes", type=int, default=1 << 19)
    p.add_argument("--kta", type=float, default=20.0)
    p.add_argument("--nrhs", type=int, default=1000)
    p.add_argument("--eps", type=float, default=1e-9)
    p.add_argument("--leaf", type=int, default=64)
    p.add_argument("--top", type=int, default=1)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--ir-tol", type=float, default=1e-8)
    p.add_argument("--sweep-fp64-levels", type=int, default=-1)
    p.add_argument("--merge", default="c64", choices=["c64", "fp64"],
                   help="mixed: merge the complex64 levels in complex64 (default) or FP64")
    p.add_argument("--merge-c64-levels", type=int, default=0,
                   help="with --merge c64: merge only the lowest N complex64 levels in complex64 (0: all)")
    p.add_argument("--tol-decay", type=float, default=0.5,
                   help="ID tolerance eps at the leaves, eps * decay^(L-l) at level l (1: the paper's single eps)")
    p.add_argument("--autotune", action="store_true", help="GEMM tile shapes from the autotuner (tuned in warm-up)")
    p.add_argument("--fw-engine", default="tensor", choices=["ff", "tensor"],
                   help="mixed: the refinement's forward operator (leaf, sibling and interpolation blocks) on the "
                        "tensor cores (default, six bf16 slices per FP64 operand) or as double-float products (ff)")
    p.add_argument("--c64-engine", default="simt", choices=["tensor", "simt"],
                   help="complex64 products on the tensor cores (bf16 pieces) or the FP32 pipe")
    p.add_argument("--sweep-ff", type=int, default=1, choices=[0, 1, 2],
                   help="mixed sweep: 1 double-float upper levels, 2 double-float everywhere")
    p.add_argument("--rank", default="learned", choices=["learned", "adaptive"],
                   help="learned (default): the trained rank network sizes a sketched ID, with the adaptive "
                        "CPQR as fallback; adaptive: the CPQR alone.  The plain FP64 comparison step always "
                        "uses the adaptive CPQR")
    p.add_argument("--workload", default="star", choices=["star", "batch64", "cgemm", "field", "omega", "mr2005"],
                   help="star: the 2^19-node star cavity (default); batch64: 64 seeded cavities of "
                        "2^12-2^15 nodes, k_T a in [1, 20], 16 waves each, built and solved as one batch; "
                        "cgemm: the batched complex64 GEMM stage alone (--gemm-batch products of "
                        "128 x 128 by 128 x --nrhs, the leaf shape of the sweep) on both engines; "
                        "field: the displacement off the boundary (eq. integ_rep) at --field-points points "
                        "for 16 waves of the star cavity, direct and proxy-compressed; "
                        "omega: the tripod of Sec. 8 swept over omega with and without the Burton-Miller term "
                        "(wave intensity at (1, 0), Fig. wave_intensity; time per omega, Fig. omega_time); "
                        "mr2005: build and solve of the LU variant against the Woodbury form of the original "
                        "Martinsson-Rokhlin method (FP64, the default star cavity)")
    p.add_argument("--field-points", type=int, default=64, help="field: observation points")
    p.add_argument("--omega-nodes", type=int, default=6400, help="omega: tripod nodes")
    p.add_argument("--omega-max", type=float, default=40.0, help="omega: largest angular frequency")
    p.add_argument("--omega-step", type=float, default=0.05, help="omega: frequency step")
    p.add_argument("--gemm-batch", type=int, default=8192, help="cgemm: number of products")
    p.add_argument("--streams", type=int, default=8, help="batch64: concurrent cavity streams")
    p.add_argument("--no-graph", action="store_true", help="batch64: launch the solve sweeps kernel by kernel "
                   "instead of replaying their CUDA graphs")
    p.add_argument("--no-compare", action="store_true",
                   help="skip the plain-FP64 comparison step (error and timings of the FP64 solver)")
    return p.parse_args()


# forward-operator phases on the tensor cores with --fw-engine tensor, and
# their algorithmic flops per column
TENSOR_FW = {"a7.fw_leaf_diag": "8 d^2 per leaf", "a7.fw_sibling": "8 x 2 r_a r_b per parent",
             "a7.fw_interp_up": "8 k (n - k) per cell and component",
             "a7.fw_interp_down": "8 k (n - k) per cell and component"}


def max_over_ranks(value, device):
    """The largest of the ranks' values (the job's time is its slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(args, rank):
    import workloads
    xy = workloads.star(args.nodes, 0.2, 5, rot=0.013 * rank)
    omega = workloads.omega_for_kTa(args.kta)
    kinds, angles = workloads.plane_wave_set(args.nrhs // 2)
    return xy, omega, kinds, angles


# ---------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                v = [x.strip() for x in line.split(",")]
                if len(v) < 9:
                    continue
                try:
                    rows.append(dict(sm=float(v[1]), smax=float(v[2]), hw=v[5], hwt=v[6], swt=v[7], pcap=v[8]))
                except ValueError:
                    continue
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = sorted(r["sm"] for r in rows)
        reasons = set()
        for r in rows:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                            ("pcap", "sw_power_cap")):
                if r[k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": rows[0]["smax"], "reasons": sorted(reasons),
                "samples": len(rows)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def phase_on_fp32(name, precision, merge_c64=False):
    """Whether a phase's arithmetic runs on the FP32 pipe: the mixed solve's
    sweep levels (complex64 and double-float), the refinement's double-float
    forward operator and, with complex64 merges, the merges (their complex64
    levels hold most of the merge flops; the upper levels stay FP64);
    everything else (quadrature, CPQR, top LU and top solve) is FP64."""
    if precision != "mixed":
        return False
    return ((name.startswith("a6.") and name != "a6.top_solve") or name.startswith("a7.")
            or (merge_c64 and name.startswith("a3.")))


# ---------------------------------------------------------------- oracle (CPU)
def oracle_sample(args, n_sample, nrhs_sample):
    """Time the oracle ('Conv': dense Galerkin assembly + LU + back substitution)
    on the same cavity shape and frequency with n_sample nodes; extrapolate to
    the full job as O(N^2) assembly + O(N^3) LU + O(N^2) per right-hand side."""
    import workloads
    from oracle import bem
    xy = workloads.star(n_sample, 0.2, 5)
    omega = workloads.omega_for_kTa(args.kta)
    P = bem.phys(2.0, 1.0, 1.0, omega)
    t0 = time.perf_counter()
    A = bem.dense_matrix(P, xy)
    t1 = time.perf_counter()
    import scipy.linalg as sl
    lu = sl.lu_factor(A, check_finite=False)
    t2 = time.perf_counter()
    F = np.stack([bem.rhs(P, xy, k % 2, 0.1 * k) for k in range(nrhs_sample)], 1)
    t3 = time.perf_counter()
    sl.lu_solve(lu, F, check_finite=False)
    t4 = time.perf_counter()
    s = args.nodes / n_sample
    t_asm, t_lu, t_rhs = t1 - t0, t2 - t1, (t4 - t2) / nrhs_sample
    full = t_asm * s ** 2 + t_lu * s ** 3 + args.nrhs * t_rhs * s ** 2
    return dict(full_s=full, t_asm=t_asm, t_lu=t_lu, t_per_rhs=t_rhs, wall=t4 - t0,
                sample="star 1+0.2cos5t, %d nodes (%d unknowns), k_T a=%g, dense assembly %.2fs + LU %.2fs + "
                       "%d RHS %.3fs; extrapolated to %d nodes x %d RHS by O(N^2) assembly, O(N^3) LU, "
                       "O(N^2) per RHS" % (n_sample, 2 * n_sample, args.kta, t_asm, t_lu, nrhs_sample,
                                           t4 - t3 + (t3 - t2), args.nodes, args.nrhs))


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return
    from oracle import build as ob
    ob.build()
    cores = os.cpu_count()
    # the sample of the bench's cpu_baseline leg (1024 nodes, 8 waves): large
    # enough that the LU time follows its O(N^3) law, a few seconds per step
    n_s = 1024
    for _ in range(args.warmup):
        oracle_sample(args, n_s, 8)
    vals = []
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = oracle_sample(args, n_s, 8)
        vals.append(last["full_s"])
    wall = time.perf_counter() - t0
    v = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / max(args.steps, 1),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic",
            "config": {"workload": "star r=1+0.2cos5t, %d nodes (2^20 unknowns), k_T a=%g, %d plane P/SV waves"
                                   % (args.nodes, args.kta, args.nrhs), "kind": "oracle dense Galerkin + LU (CPU)"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle", "sample": last["sample"]},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- batched cavities
def run_cgemm(args, fds, torch, rank):
    """Stage benchmark of the batched complex64 GEMM: nb products of
    128 x 128 by 128 x n (seeded normal entries), each engine timed with CUDA
    events over --steps calls after --warmup, and its normwise error on eight
    products against the complex128 product of the same inputs."""
    import numpy as np
    nb, d, n = args.gemm_batch, 128, args.nrhs
    g = torch.Generator(device="cuda")
    g.manual_seed(1 + rank)
    A = torch.randn(nb * d * d * 2, device="cuda", generator=g)
    B = torch.randn(nb * d * n * 2, device="cuda", generator=g)
    aoff = np.arange(nb, dtype=np.int64) * d * d
    boff = np.arange(nb, dtype=np.int64) * d * n
    out = {}
    for name, eng in (("tensor", fds.FDS_C64_TENSOR), ("simt", fds.FDS_C64_SIMT)):
        C = torch.zeros(nb * d * n * 2, device="cuda")
        call = lambda: fds.fds_cgemm_c64_batched([d] * nb, [n] * nb, [d] * nb, aoff, boff, boff, A, B, C,
                                                 engine=eng)
        for _ in range(args.warmup):
            call()
        ts = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            call()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        Ah, Bh, Ch = A.view(-1, 2).cpu().numpy(), B.view(-1, 2).cpu().numpy(), C.view(-1, 2).cpu().numpy()
        err = 0.0
        for b in range(0, nb, max(1, nb // 8)):
            cp = lambda X, o, r, c: (X[o:o + r * c, 0] + 1j * X[o:o + r * c, 1]).reshape(c, r).T
            a = cp(Ah, b * d * d, d, d).astype(np.complex128)
            x = cp(Bh, b * d * n, d, n).astype(np.complex128)
            ref = a @ x
            got = cp(Ch, b * d * n, d, n)
            err = max(err, float(np.max(np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0))))
        ms = float(np.median(ts))
        out[name] = {"ms": ms, "tflops_complex": 8.0 * nb * d * d * n / ms / 1e9, "max_rel_err": err}
    if rank == 0:
        print(json.dumps({"workload": "cgemm %d x (128 x 128) x (128 x %d) complex64" % (nb, n),
                          "steps": args.steps, "warmup": args.warmup, "engines": out}))


def run_field(args, fds, torch, rank):
    """Field evaluation off the boundary (eq. integ_rep): the star cavity of
    the default workload is built (mixed) and solved for 16 waves (8 P + 8 SV)
    on the device; then fds_field at --field-points points on circles of radius
    1.5-3 is timed with CUDA events over --steps calls after --warmup.
    Unit: quadrature sums per second (point x element x wave)."""
    import workloads
    N = args.nodes
    xy = workloads.star(N)
    omega = workloads.omega_for_kTa(args.kta)
    kinds, angles = workloads.plane_wave_set(8)
    h = fds.fds_build(xy, omega, 2.0, 1.0, args.eps, leaf_size=args.leaf, top_level=args.top,
                      precision=fds.FDS_MIXED, ir_tol=args.ir_tol)
    F = fds.fds_rhs_plane_wave(h, kinds, angles)
    d = torch.tensor(np.ascontiguousarray(F.T), device="cuda")
    fds.fds_solve_device(h, d)
    npts = args.field_points
    rng = np.random.default_rng(7 + rank)
    r, th = rng.uniform(1.5, 3.0, npts), rng.uniform(0, 2 * np.pi, npts)
    pts = np.stack([r * np.cos(th), r * np.sin(th)], 1)
    def timed(compressed):
        for _ in range(args.warmup):
            fds.fds_field(h, d, kinds, angles, pts, compressed=compressed)
        ts = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            out = fds.fds_field(h, d, kinds, angles, pts, compressed=compressed)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts)), out

    ms, ref = timed(False)
    ms_c, got = timed(True)
    err_c = float(np.abs(got - ref).max() / np.abs(ref).max())
    h.close()
    sums = float(npts) * N * len(kinds)
    if rank == 0:
        print(json.dumps({"metric": "field off the boundary (eq. integ_rep): quadrature sums per second",
                          "value": sums / ms / 1e6, "unit": "Gsum/s", "ms_per_step": ms, "steps": args.steps,
                          "warmup": args.warmup, "higher_is_better": True, "data": "synthetic",
                          "config": {"workload": "star r=1+0.2cos5t, %d nodes, k_T a=%g, %d waves, %d points, "
                                                 "8 Gauss points per element, direct summation"
                                                 % (N, args.kta, len(kinds), npts)},
                          "compressed": {"ms": ms_c, "speedup_vs_direct": ms / ms_c,
                                         "max_rel_diff_vs_direct": err_c,
                                         "note": "tree skeletons as equivalent sources (fds_field_compressed); "
                                                 "same points and waves"}}))


def run_omega(args, fds, torch, rank):
    """The tripod of Sec. 8 (lambda = mu = 1, rho = 1, leaf 100, l0 = 1,
    eps 1e-8) swept over omega = step .. --omega-max: each omega is built and
    solved with the Burton-Miller formulation (the solver's default alpha) and
    without it (alpha = 0, eq. bie_non_bie) for one plane P wave at angle 0;
    the wave intensity |u_1|^2 + |u_2|^2 at x = (1, 0), which is node 0 of the
    tripod, is recorded for both (Fig. wave_intensity), and the device time of
    build + solve per omega (Fig. omega_time)."""
    import workloads
    N = args.omega_nodes
    xy = workloads.tripod(N)
    ws = np.arange(args.omega_step, args.omega_max + 0.5 * args.omega_step, args.omega_step)
    kinds, angles = np.array([0], np.int32), np.array([0.0])
    out = {"bm": [], "non_bm": [], "ms_bm": []}
    for _ in range(args.warmup):
        h = fds.fds_build(xy, float(ws[0]), 1.0, 1.0, 1e-8, leaf_size=100, top_level=1)
        h.close()
    t0 = time.perf_counter()
    for w in ws:
        for name, alpha in (("bm", None), ("non_bm", 0.0)):
            h = fds.fds_build(xy, float(w), 1.0, 1.0, 1e-8, leaf_size=100, top_level=1, alpha=alpha,
                              tol_decay=args.tol_decay)
            x = fds.fds_solve(h, fds.fds_rhs_plane_wave(h, kinds, angles))
            st = fds.fds_stats_get(h)
            h.close()
            out[name].append(float(abs(x[0, 0]) ** 2 + abs(x[N, 0]) ** 2))
            if name == "bm":
                out["ms_bm"].append(st.build_ms + st.solve_ms)
    wall = time.perf_counter() - t0
    bm, nb = np.array(out["bm"]), np.array(out["non_bm"])
    dev = np.abs(nb - bm) / bm
    # a spike: the non-BM intensity more than 10% off the BM one
    spikes = [round(float(w), 3) for w, d in zip(ws, dev) if d > 0.1]
    # smoothness of the BM curve: largest jump relative to its neighbours' mean
    mid = 0.5 * (bm[:-2] + bm[2:])
    bm_jump = float(np.max(np.abs(bm[1:-1] - mid) / mid)) if len(bm) > 2 else 0.0
    ms = np.array(out["ms_bm"])
    if rank == 0:
        print(json.dumps({"metric": "omega sweep: build + solve per omega (tripod, Sec. 8.4)",
                          "value": float(np.median(ms)), "unit": "ms", "higher_is_better": False,
                          "data": "synthetic", "warmup": args.warmup, "wall_s": wall,
                          "config": {"workload": "tripod (Sec. 8, Fig. tripod), %d nodes, lambda=mu=1, rho=1, leaf 100, "
                                                 "l0=1, eps 1e-8, tol_decay %g, one plane P wave at 0, omega %g..%g "
                                                 "step %g" % (N, args.tol_decay, ws[0], ws[-1], args.omega_step)},
                          "ms_per_omega_by_range": {"%g-%g" % (a, b): float(np.median(ms[(ws >= a) & (ws < b)]))
                                                    for a, b in ((0, 10), (10, 20), (20, 30), (30, 41))
                                                    if np.any((ws >= a) & (ws < b))},
                          "non_bm_spikes": spikes, "non_bm_spike_count": len(spikes),
                          "max_rel_dev_non_bm_vs_bm": float(dev.max()),
                          "bm_max_rel_jump": bm_jump,
                          "omega": [round(float(w), 4) for w in ws],
                          "intensity_bm": [float("%.6g" % v) for v in bm],
                          "intensity_non_bm": [float("%.6g" % v) for v in nb]}))


def run_mr2005(args, fds, torch, rank):
    """The paper's LU-based variant against the Woodbury form of the original
    Martinsson-Rokhlin method (FDS_VARIANT_MR2005), both plain FP64 on the
    default star cavity: build time, the build's matrix-matrix work (flops of
    the merge phases), per-RHS solve time, and the relative difference of the
    two solutions (same skeletons: rounding only)."""
    import workloads
    xy = workloads.star(args.nodes)
    omega = workloads.omega_for_kTa(args.kta)
    kinds, angles = workloads.plane_wave_set(args.nrhs // 2)
    res, sols = {}, {}
    for name, var in (("lu", fds.FDS_VARIANT_LU), ("mr2005", fds.FDS_VARIANT_MR2005)):
        for it in range(args.warmup + 1):
            fds.fds_timing_reset()
            fds.fds_timing_enable(it == args.warmup)
            h = fds.fds_build(xy, omega, 2.0, 1.0, args.eps, leaf_size=args.leaf, top_level=args.top,
                              tol_decay=args.tol_decay, variant=var)
            d = torch.empty((len(kinds), 2 * args.nodes), dtype=torch.complex128, device="cuda")
            fds.fds_rhs_plane_wave_device(h, torch.from_numpy(kinds).cuda(), torch.from_numpy(angles).cuda(), d)
            fds.fds_solve_device(h, d)
            torch.cuda.synchronize()
            fds.fds_timing_enable(False)
            st = fds.fds_stats_get(h)
            h.close()
        rep = fds.fds_timing_report()
        res[name] = {"build_s": st.build_ms / 1e3, "per_rhs_us": st.solve_ms * 1e3 / len(kinds),
                     "factor_gb": st.factor_bytes / 1e9,
                     "merge_gflop": sum(v["flops"] for k, v in rep.items() if k.startswith("a3.")) / 1e9,
                     "merge_ms": sum(v["ms"] for k, v in rep.items() if k.startswith("a3.")),
                     "sweep_gflop": sum(v["flops"] for k, v in rep.items() if k.startswith("a6.")) / 1e9}
        sols[name] = d
    err = (torch.linalg.vector_norm(sols["mr2005"] - sols["lu"], dim=1) /
           torch.linalg.vector_norm(sols["lu"], dim=1)).max().item()
    if rank == 0:
        print(json.dumps({"metric": "LU variant vs Woodbury (MR2005) form: build s, merge GFLOP, per-RHS us",
                          "value": res["mr2005"]["build_s"] / res["lu"]["build_s"], "unit": "build time ratio "
                          "MR2005 / LU", "higher_is_better": False, "data": "synthetic", "warmup": args.warmup,
                          "config": {"workload": "star r=1+0.2cos5t, %d nodes, k_T a=%g, eps %g, tol_decay %g, "
                                                 "leaf %d, %d waves, FP64" % (args.nodes, args.kta, args.eps,
                                                                              args.tol_decay, args.leaf, len(kinds))},
                          "lu": res["lu"], "mr2005": res["mr2005"], "max_rel_diff": err}))


def run_batch(args, fds, torch, world, rank, local):
    """64 seeded cavities (ellipses / stars, 2^12..2^15 nodes, k_T a in [1, 20],
    eps 1e-8, leaf 64, complex128 as in the batched configuration) built
    with fds_build_batch on --streams concurrent streams, 16 plane waves each
    (8 P + 8 SV), solved with one launch per tree level and phase across the
    cavities (fds_solve_batch_levels; CUDA-graph replay unless --no-graph).
    One step = batch build + load vectors + batch solve; after the timed
    steps the same work one cavity at a time (1 stream) is timed once, and
    the solve alone of one built batch both ways (level-batched launches,
    per-cavity streams)."""
    import workloads
    cav = workloads.random_cavities(64, seed=workloads.SEED + 2 + 97 * rank)
    for c in cav:
        c["omega"] = workloads.omega_for_kTa(c["kTa"])
    kinds, angles = workloads.plane_wave_set(8)
    d_k = torch.from_numpy(kinds).cuda()
    d_a = torch.from_numpy(angles).cuda()
    d_F = [torch.empty((16, 2 * c["N"]), dtype=torch.complex128, device="cuda") for c in cav]
    eps = 1e-8
    prec = fds.FDS_FP64
    stream = torch.cuda.Stream()

    def load(hs):
        for h, F in zip(hs, d_F):
            fds.fds_rhs_plane_wave_device(h, d_k, d_a, F, fds.fds_handle_stream(h))

    def solve(hs, levels, graph, streams):
        if levels:
            with torch.cuda.stream(stream):
                fds.fds_solve_batch_levels(hs, d_F, use_graph=graph, stream=stream.cuda_stream)
        else:
            fds.fds_solve_batch(hs, d_F, n_streams=streams)

    def step(streams, graph=not args.no_graph, levels=True):
        hs = fds.fds_build_batch(cav, 2.0, 1.0, eps, n_streams=streams, leaf_size=args.leaf, precision=prec,
                                 use_graph=graph)
        load(hs)
        solve(hs, levels and streams > 1, graph, streams)
        for h in hs:
            h.close()

    for _ in range(args.warmup):
        step(args.streams)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = fds.fds_launch_count()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(args.streams)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / args.steps
    launches = (fds.fds_launch_count() - launches0) // args.steps
    clk = clocks.stop()
    ms = max_over_ranks(ms, "cuda")
    t1 = time.perf_counter()
    step(1)
    torch.cuda.synchronize()
    seq_ms = (time.perf_counter() - t1) * 1e3
    # the solve alone of one built batch: level-batched launches (graph and
    # plain) against per-cavity streams, best of three each
    hs = fds.fds_build_batch(cav, 2.0, 1.0, eps, n_streams=args.streams, leaf_size=args.leaf, precision=prec)
    solve_ms, solve_launches = {}, {}
    for name, levels, graph in (("levels_graph", True, True), ("levels", True, False), ("streams", False, False)):
        best = None
        for _ in range(3):
            load(hs)
            torch.cuda.synchronize()
            l0_ = fds.fds_launch_count()
            t = time.perf_counter()
            solve(hs, levels, graph, args.streams)
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t) * 1e3
            best = dt if best is None else min(best, dt)
            solve_launches[name] = int(fds.fds_launch_count() - l0_)
        solve_ms[name] = best
    for h in hs:
        h.close()
    if rank != 0:
        return
    nodes = sum(c["N"] for c in cav)
    line = {"metric": "batched build + solve of 64 cavities (s per batch)", "value": ms / 1e3, "unit": "s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128", "data": "synthetic",
            "config": {"workload": "64 seeded cavities (ellipse aspect 1-4 / star e in [0,0.3], m in 3..8), "
                                   "2^12-2^15 nodes (%d in total), k_T a in [1,20], eps 1e-8, leaf %d, "
                                   "16 plane waves each, complex128, build on %d streams, solve with one "
                                   "launch per level and phase across the cavities" % (nodes, args.leaf,
                                                                                        args.streams),
                       "timing": "host wall clock around the whole batch (several streams), synchronised"},
            "sequential_ms": seq_ms, "speedup_vs_sequential": seq_ms / ms, "gpu_launches": int(launches),
            "graph": not args.no_graph, "solve_only_ms": solve_ms, "solve_only_launches": solve_launches,
            "clocks": clk}
    print(json.dumps(line))


# ---------------------------------------------------------------- ours
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    world, rank, local = dist_setup()
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__ as g
    g.build()
    from paper_2411_18026_gb300 import fds
    if args.workload == "batch64":
        run_batch(args, fds, torch, world, rank, local)
        return
    if args.workload == "cgemm":
        run_cgemm(args, fds, torch, rank)
        return
    if args.workload == "field":
        run_field(args, fds, torch, rank)
        return
    if args.workload == "omega":
        run_omega(args, fds, torch, rank)
        return
    if args.workload == "mr2005":
        run_mr2005(args, fds, torch, rank)
        return
    if args.autotune:
        fds.fds_autotune_enable(True)

    xy, omega, kinds, angles = workload(args, rank)
    N = len(xy)
    stream = torch.cuda.current_stream()
    d_kinds = torch.from_numpy(kinds).cuda()
    d_angles = torch.from_numpy(angles).cuda()
    d_F = torch.empty((args.nrhs, 2 * N), dtype=torch.complex128, device="cuda")

    info = {}

    prec = fds.FDS_MIXED if args.precision == "mixed" else fds.FDS_FP64
    from paper_2411_18026_gb300 import learned
    mlp = learned.load_params() if args.rank == "learned" else None
    rank_used = "learned" if mlp is not None else "adaptive"
    c64_engine = fds.FDS_C64_TENSOR if args.c64_engine == "tensor" else fds.FDS_C64_SIMT

    def step(precision=prec, out=d_F, rec=info, params=mlp):
        h = fds.fds_build(xy, omega, 2.0, 1.0, args.eps, leaf_size=args.leaf, top_level=args.top, stream=stream,
                          precision=precision, ir_tol=args.ir_tol, sweep_fp64_levels=args.sweep_fp64_levels,
                          mlp_params=params, merge_c64=args.merge == "c64" and precision == fds.FDS_MIXED,
                          fw_engine=fds.FDS_FW_TENSOR if args.fw_engine == "tensor" and precision == fds.FDS_MIXED
                          else fds.FDS_FW_FF,
                          tol_decay=args.tol_decay, merge_c64_levels=args.merge_c64_levels,
                          sweep_ff=args.sweep_ff if precision == fds.FDS_MIXED else 0,
                          c64_engine=c64_engine)
        fds.fds_rhs_plane_wave_device(h, d_kinds, d_angles, out, stream)
        rec["converged"] = True
        try:
            fds.fds_solve_device(h, out, stream)
        except fds.FdsError as e:
            if e.code != fds.FDS_ERR_NOT_CONVERGED:
                raise
            rec["converged"] = False
        st = fds.fds_stats_get(h)
        rec["build_ms"], rec["solve_ms"] = st.build_ms, st.solve_ms
        rec["top_size"], rec["levels"] = st.top_size, st.levels
        rec["factor_gb"] = st.factor_bytes / 1e9
        rec["skeleton_dofs"] = [int(st.skeleton_dofs[l]) for l in range(st.levels + 1)]
        rec["ir_iters"], rec["ir_residual"] = st.ir_iters, st.ir_residual
        rec["id_sketched"], rec["id_fallback"] = st.id_sketched, st.id_fallback
        h.close()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # roofline denominators of the FP64 and FP32 phases, measured on this GPU
    alu_peaks = {"fp64_tflops": fds.fds_alu_peak(0), "fp32_tflops": fds.fds_alu_peak(1),
                 "sms": torch.cuda.get_device_properties(local).multi_processor_count}
    fds.fds_timing_reset()
    fds.fds_timing_enable(True)
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = fds.fds_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    builds, solves = [], []
    for _ in range(args.steps):
        step()
        builds.append(info["build_ms"])
        solves.append(info["solve_ms"])
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    launches = (fds.fds_launch_count() - launches0) // args.steps
    clk = clocks.stop()
    fds.fds_timing_enable(False)
    phases = fds.fds_timing_report()
    ms = max_over_ranks(ms, "cuda")

    # plain-FP64 comparison on the same inputs (outside the timed region)
    compare = None
    if args.precision == "mixed" and not args.no_compare and rank == 0:
        d_F64 = torch.empty_like(d_F)
        rec = {}
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        step(fds.FDS_FP64, d_F64, rec, None)
        c1.record(stream)
        torch.cuda.synchronize()
        num = torch.linalg.vector_norm(d_F - d_F64, dim=1)
        den = torch.linalg.vector_norm(d_F64, dim=1)
        err = (num / den).max().item()
        compare = {"fp64_ms_per_step": c0.elapsed_time(c1), "fp64_build_s": rec["build_ms"] / 1e3,
                   "fp64_per_rhs_us": rec["solve_ms"] * 1e3 / args.nrhs, "fp64_factor_gb": rec["factor_gb"],
                   "max_rel_err_vs_fp64": err,
                   "note": "max over the right-hand sides of ||x_mixed - x_fp64|| / ||x_fp64||"}
        del d_F64

    # end to end through the host-buffer C ABI: geometry and right-hand sides
    # from pinned host memory, solution back to pinned host memory
    e2e = None
    if not args.no_e2e:
        F_host = torch.empty((args.nrhs, 2 * N), dtype=torch.complex128, pin_memory=True)
        F_host.copy_(d_F)     # (values are irrelevant for timing; any RHS of the right size)
        F_np = F_host.numpy()
        xy_host = torch.from_numpy(np.ascontiguousarray(xy)).pin_memory().numpy()
        import ctypes
        L = fds.lib()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g_ = fds.fds_geometry(N, xy_host.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1.0)
        o = fds.default_options()
        o.leaf_size, o.top_level = args.leaf, args.top
        o.precision, o.ir_tol, o.sweep_fp64_levels = prec, args.ir_tol, args.sweep_fp64_levels
        o.merge_c64 = 1 if args.merge == "c64" and prec == fds.FDS_MIXED else 0
        o.merge_c64_levels = args.merge_c64_levels
        o.tol_decay = args.tol_decay
        o.fw_engine = fds.FDS_FW_TENSOR if args.fw_engine == "tensor" and prec == fds.FDS_MIXED else fds.FDS_FW_FF
        o.sweep_ff = args.sweep_ff
        o.c64_engine = c64_engine
        mlp32 = None
        if mlp is not None:
            mlp32 = np.ascontiguousarray(mlp, dtype=np.float32)
            o.rank_mode = fds.FDS_RANK_LEARNED
            o.mlp_params = mlp32.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        out = ctypes.c_void_p()
        rc = L.fds_build_ex(ctypes.byref(g_), float(omega), 2.0, 1.0, float(args.eps), ctypes.byref(o),
                            ctypes.byref(out))
        assert rc == 0, rc
        rc = L.fds_solve(out, F_np.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double)), args.nrhs)
        assert rc in (fds.FDS_OK, fds.FDS_ERR_NOT_CONVERGED), rc
        L.fds_destroy(out)
        t_e2e = time.perf_counter() - t0
        e2e = {"value": t_e2e * world / world, "unit": "s", "h2d_bytes_per_step": int(xy_host.nbytes + F_np.nbytes),
               "d2h_bytes_per_step": int(F_np.nbytes)}
        del F_host

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # FP64 flops and DRAM bytes per quadrature point of the kernel-evaluation
    # kernels, from ncu counters (dfma x 2 + dmul + dadd; dram read + write)
    # over the launches of one 2^14-node build of the same cavity: executed
    # FP64 operations of the evaluator, so the fraction below is the FP64
    # pipe's use by the quadrature
    A1_PER_POINT = {"a1.leaf_blocks": (475.0, 0.66), "a1.near_rows": (493.0, 1.54), "a1.proxy_rows": (493.0, 1.54),
                    "a1.sibling_blocks": (509.0, 0.18), "a1.top_blocks": (509.0, 0.18)}
    pk, src = peaks()
    alu = alu_peaks
    roof, per_phase = None, {}
    for name, d in sorted(phases.items()):
        if d["ms"] <= 0:
            continue
        launches_ = max(d["launches"], 1)
        flops, traffic, basis = d["flops"], None, "algorithmic flop count of the phase (library)"
        if name in A1_PER_POINT and d["units"] > 0:
            fpp, bpp = A1_PER_POINT[name]
            flops = d["units"] * fpp
            traffic = d["units"] * bpp / launches_
            basis = ("quadrature points x %.0f executed FP64 flops per point (ncu, 2^14-node build); traffic = points "
                     "per launch x %.2f DRAM bytes per point (same capture)" % (fpp, bpp))
        fp32 = phase_on_fp32(name, args.precision, args.merge == "c64")
        peak = alu["fp32_tflops"] if fp32 else alu["fp64_tflops"]
        pipe, bound = "fp32" if fp32 else "fp64", "alu"
        if name in TENSOR_FW and args.fw_engine == "tensor" and args.precision == "mixed":
            # 21 bf16 slice products per FP64-accurate product, on the tensor cores
            flops, pipe, bound = 21.0 * flops, "tensor (bf16)", "tensor"
            peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1900.0))
            basis = "21 bf16 products x the phase's algorithmic flops (%s)" % TENSOR_FW[name]
        ent = {"ms_per_step": d["ms"] / args.steps, "launches_per_step": d["launches"] / args.steps,
               "bound": bound, "pipe": pipe, "basis": basis}
        if flops > 0:
            ach = flops / (d["ms"] / 1e3) / 1e12
            ent.update(achieved_tflops=ach, peak_tflops=peak, frac=ach / peak)
        if d["bytes"] > 0:
            gbs = d["bytes"] / (d["ms"] / 1e3) / 1e9
            ent.update(achieved_gbs=gbs, hbm_frac=gbs / pk["hbm_gbs"])
            if flops <= 0 or gbs / pk["hbm_gbs"] > ent.get("frac", 0):
                ent["bound"] = "hbm"
        if d["units"] > 0:
            ent["quad_points_per_s"] = d["units"] / (d["ms"] / 1e3)
        per_phase[name] = ent
        # a7.forward_apply brackets its a7.fw_* parts: not a kernel of its own
        if name == "a7.forward_apply":
            ent["note"] = "sum of the a7.fw_* phases"
            continue
        if roof is None or d["ms"] > roof["_ms"]:
            roof = {"_ms": d["ms"], "kernel": name, "bound": ent["bound"], "achieved": ent.get("achieved_tflops"),
                    "peak": peak, "unit": "TFLOP/s", "frac": ent.get("frac"), "traffic": traffic,
                    "peak_source": ("MEASURED_PEAKS.json bf16 (sustained), %s" % src) if bound == "tensor" else
                                   "measured on this GPU before the timed steps (fds_alu_peak: FMA loop, %s pipe, "
                                   "%d SMs)" % ("FP32" if fp32 else "FP64", alu["sms"]),
                    "basis": basis, "avg_launch_ms": d["ms"] / launches_,
                    "launches_per_step": d["launches"] / args.steps}
    if roof:
        roof.pop("_ms")

    cpu = None
    if not args.no_cpu:
        from oracle import build as ob
        ob.build()
        smp = oracle_sample(args, 1024, 8)
        cpu = {"value": smp["full_s"], "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": smp["sample"]}
    build_s = float(np.median(builds)) / 1e3
    per_rhs_us = float(np.median(solves)) * 1e3 / args.nrhs
    line = {
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128+c64" if args.precision == "mixed" else "c128", "data": "synthetic",
        "config": {"workload": "star r=1+0.2cos5t, %d nodes (%d complex unknowns), lambda=2 mu=1 rho=1, "
                               "k_T a=%g, leaf %d, l0=%d, eps=%g (leaf level; x%g per level up), %d plane P/SV "
                               "waves, %s"
                               % (N, 2 * N, args.kta, args.leaf, args.top, args.eps, args.tol_decay, args.nrhs,
                                  ("mixed precision (%s merges of the complex64 levels), refined to residual %g"
                                   % (args.merge, args.ir_tol) if args.precision == "mixed" else "plain FP64")
                                  + ", %s rank" % rank_used),
                   "l2": "working set (factors, vectors) larger than L2; no flush",
                   "precision": args.precision, "c64_engine": args.c64_engine, "merge": args.merge,
                   "merge_c64_levels": args.merge_c64_levels,
                   "tol_decay": args.tol_decay, "autotune": bool(args.autotune), "fw_engine": args.fw_engine,
                   "fp64_reference": "plain FP64 build (adaptive CPQR, same eps and tol_decay) on the same inputs"},
        "ir_iters": info.get("ir_iters"), "ir_residual": info.get("ir_residual"),
        "ir_converged": info.get("converged"), "vs_fp64": compare, "rank_mode": rank_used,
        "id_sketched": info.get("id_sketched"), "id_fallback": info.get("id_fallback"),
        "build_s": build_s, "per_rhs_us": per_rhs_us,
        "levels": info.get("levels"), "top_size": info.get("top_size"), "factor_gb": info.get("factor_gb"),
        "skeleton_dofs": info.get("skeleton_dofs"),
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "roofline": roof, "cpu_baseline": cpu,
        "alu_peaks": alu, "phases_roofline": per_phase,
        "quad_points_per_step": {k: v["units"] / args.steps for k, v in sorted(phases.items()) if v["units"] > 0},
    }
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
