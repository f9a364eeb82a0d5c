"""Benchmark: time to a 1e-3 relative (1 sigma) MG-MLMC++ estimate of tr(D^{-1}).

One step = the whole hot path on one synthetic gauge field already resident
in HBM: multigrid set-up (test vectors, aggregation, Galerkin stencils,
coarsest inverse), the Hutch++ sketches of every level difference and the
stochastic loop of Algorithm 2 until the relative accuracy eps is reached.
Workload (default): L = 512 (n = 524288), beta = 5, m0 tuned so that the
smallest |eigenvalue| of D is ~1e-3, 4 levels (512 -> 128 -> 32 -> 8), 4x4
aggregates, 8 test vectors per chirality, d = 32, k = 2, up to 256 rhs per
batch, eps = 1e-3, mixed precision (FP32 inner FGMRES + V-cycle, FP64 true
residual refinement to 1e-10, FP64 sketch/projection/statistics).

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample instead.  Multi-GPU runs are independent replicas (one field
per rank, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# V(2,2): of V(1,1) .. V(4,4), K-cycles and bootstrap 1-3 measured on this workload, the fastest set-up + estimate.
# tensor_cores = 3: FP16 coarse-level tensor-core operands (11-bit significands like TF32; the stencil runs the
# 2x2-block kernel where the tuner finds it faster); measured 0.841 s against 0.843 s with TF32 (= 2) and 0.844 s
# with BF16 (= 1).
# autotune = 1: launch variants timed in the first set-up (a warm-up step) and reused from the tuning table.
# First batch of 8 samples per level (then batches sized from the variances, up to 256): the stop rule needs 6-8
# samples on levels 0 and 1 here, so a first batch of 16 only computed samples that are discarded.
# Sketch d = 32, k = 2 (the workload's configuration).  A d x k scan on this workload finds smaller sketches faster
# (the deflated part removes little variance on these fields); the benchmark line also reports one estimate with
# d = 16, k = 1 (32 difference-operator applications per level) as `sketch_d16_k1`.
WORKLOAD = dict(L=512, beta=5.0, seed=0, ntv=8, d=32, k=2, eps=1e-3, nrhs_max=256, nrhs_first=8,
                bootstrap=2, bootstrap_its=6, kcycle_its=0, pre_smooth=2, post_smooth=2, tensor_cores=3, autotune=1)
FALLBACK_M0 = {512: -0.07, 128: -0.1199}


# DRAM bytes per algorithmic byte of the tensor-core coarse kernels, from one ncu capture each of a level-1 launch
# with 32 rhs of the L = 512 hierarchy (dram__bytes_read + _write against the launch's algorithmic bytes); the
# benchmark scales them to its average launch.  Per-site TF32 stencil: 235.99 + 48.96 MB against 301.99 MB.
# 2x2-block FP16 stencil, SAP residual of one colour: 109.31 + 5.99 MB against 109.05 MB (8192 sites x 32 rhs x
# 256 B + 41.94 MB of weights); SAP block update: 83.95 + 5.74 MB against 134.22 MB (its x and 16-bit copy
# writes stay in L2).
TRAFFIC_PER_ALG_BYTE = {
    "MODE = 0; int BF = 0": ((235.987 + 48.964) / 301.990, "ncu capture of one launch (level 1, 32 rhs): 284.95 MB "
                            "DRAM / 301.99 MB algorithmic, scaled to the average launch"),
    "k_tcb_kernel": ((109.313 + 5.991) / 109.052, "ncu capture of one SAP-residual launch (level 1, 32 rhs, FP16): "
                     "115.30 MB DRAM / 109.05 MB algorithmic, scaled to the average launch"),
    "k_tcs_kernel": ((83.952 + 5.735) / 134.218, "ncu capture of one SAP block-update launch (level 1, 32 rhs, "
                     "FP16): 89.69 MB DRAM / 134.22 MB algorithmic, scaled to the average launch"),
}


def mass_for(L: int, beta: float, seed: int) -> float:
    path = os.path.join(ROOT, "tests", "golden", "masses.json")
    try:
        data = json.load(open(path))
        return float(data["L%d_beta%g_seed%d" % (L, beta, seed)]["m0"])
    except Exception:
        return FALLBACK_M0.get(L, -0.05)


def peaks() -> dict:
    p = dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0, src="fallback")
    try:
        m = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        p.update(hbm_gbs=float(m["hbm_gbs"]), bf16_tflops=float(m["bf16_tflops"]),
                 bf16_tflops_sustained=float(m.get("bf16_tflops_sustained", m["bf16_tflops"])), src="measured")
    except Exception:
        pass
    # CUDA-core peaks from unit counts and the maximum SM clock (152 SMs x 128 FP32 lanes x 2 flops) and the
    # nominal FP64 rate; the benchmark replaces both by the library's measurement (mgmlmc_alu_peak)
    p["fp32_alu_tflops"] = 152 * 128 * 2 * 2.070e9 / 1e12
    p["fp64_alu_tflops"] = 1.25
    # dense TF32 tensor rate: the measured sustained bf16 rate times the nominal tf32 / bf16 ratio (1.1 / 2.25)
    p["tf32_tensor_tflops_sustained"] = p["bf16_tflops_sustained"] * 1.1 / 2.25
    return p


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self) -> dict:
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for i, nm in enumerate(names):
                    if r[3 + i].lower().startswith("active"):
                        reasons.add(nm)
            except Exception:
                continue
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return dict(sm_mhz=med, sm_max_mhz=mx, reasons=sorted(reasons), samples=len(sm))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_seed(base: int, rank: int) -> int:
    """Gauge-field seed of one replica: every rank estimates its own field (no data-path collective)."""
    return base + rank


def max_over_ranks(x: float, world: int, device="cuda") -> float:
    """The largest x over the ranks of the default process group: the slowest replica sets the job's time."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle (reference arm / cpu_baseline)
# Sample counts N_l of the L = 512 GPU estimate (bench default), used by the reference arm, which runs no GPU
N_WORKLOAD_L512 = [8, 7, 58]


class OracleWorkload:
    """The CPU oracle, as it stands, on the benchmark's own L = 512 field, measured per part and extrapolated to
    the time to the target accuracy (a full oracle run takes minutes of sparse LU and hundreds of direct
    solves):
      set-up   the oracle's hierarchy (test vectors smoothed by one SAP sweep) and the sparse-LU factorization of
               every level (LevelDifference), timed once;
      batch    one batch of `nb` accumulated-form level-difference applications per level difference
               (fine-size Rademacher vectors, direct solves on levels l and l+1) with the projected sample
               zeta^H y, timed per level;
      total    set-up + sum_l t_l x ((k + 1) d + N_l): the (k + 1) d sketch and low-rank applications of
               Algorithm 2's deflation part and the N_l stochastic samples (the CholeskyQR2 and the coarsest
               dense trace are part of the set-up or negligible)."""

    def __init__(self, U_host, L, m0, seed=0):
        from oracle import estimators as oest
        from oracle import multigrid as omg
        from oracle import schwinger as osch
        W = WORKLOAD
        t0 = time.perf_counter()
        D = osch.dirac_sparse(U_host, m0)
        H = omg.Hierarchy(D, L, ntv=W["ntv"], setup_sweeps=1, seed=seed)
        self.ld = oest.LevelDifference(H)
        self.t_setup = time.perf_counter() - t0
        self.H, self.L, self.seed = H, L, seed
        self.t_sample = None

    def batch(self, nb=4):
        """seconds per level-difference sample, per level (one batch of nb)"""
        from oracle import rng as orng
        import numpy as np
        out = []
        n0 = self.H.n[0]
        for l in range(self.H.levels - 1):
            Z = orng.rademacher_block(self.seed, l, orng.PHASE_STOCH, 0, n0, nb)
            t0 = time.perf_counter()
            Y = self.ld.apply(l, Z)
            np.einsum("ij,ij->j", np.conj(Z), Y)
            out.append((time.perf_counter() - t0) / nb)
        self.t_sample = out
        return out

    def total(self, N, d, k):
        return self.t_setup + sum(t * ((k + 1) * d + n) for t, n in zip(self.t_sample, N))

    def describe(self, N, d, k, nb):
        return ("oracle (numpy/scipy FP64, sparse LU) on the L=%d beta=%g workload field: hierarchy set-up and "
                "sparse-LU factorization of all %d levels timed (%.1f s), one batch of %d level-difference samples "
                "per level timed (%s s each); time to eps extrapolated as set-up + sum_l t_l ((k+1) d + N_l) with "
                "d=%d, k=%d, N_l=%s" % (self.L, WORKLOAD["beta"], self.H.levels, self.t_setup, nb,
                                        ", ".join("%.3g" % t for t in self.t_sample), d, k, list(N)))


def run_reference(args):
    """Reference arm: the oracle on the benchmark's L = 512 workload, set-up once (its time is part of every
    step's value), then per step one batch of level-difference samples per level; value = the extrapolated time
    to eps with the workload's sample counts."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count()))
    from synthetic import gauge
    W = WORKLOAD
    L = args.L
    U = gauge.links(gauge.field(L, W["beta"], W["seed"]))
    orc = OracleWorkload(U, L, mass_for(L, W["beta"], W["seed"]), W["seed"])
    nb = 4
    vals = []
    for i in range(args.warmup + args.steps):
        orc.batch(nb)
        if i >= args.warmup:
            vals.append(orc.total(N_WORKLOAD_L512, W["d"], W["k"]))
    v = sum(vals) / len(vals)
    cores = os.cpu_count()
    sample = orc.describe(N_WORKLOAD_L512, W["d"], W["k"], nb) + " (N_l: the GPU estimate's counts)"
    line = dict(impl="reference", metric="time_to_eps_s", value=v, unit="s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * v, higher_is_better=False, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                config=dict(workload=workload_name(W, L)),
                cpu_baseline=dict(value=v, unit="s", cores=cores, kind="oracle", sample=sample),
                e2e=dict(value=v, unit="s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


def workload_name(W, L, m0=None, nlev=4):
    return ("MG-MLMC++ tr(D^-1), 2D Schwinger Wilson-Dirac, L=%d, beta=%g, m0=%.6f, %d levels, ntv=%d/chirality, "
            "d=%d, k=%d, nrhs<=%d, eps=%g, mixed FP32/FP64, solver tol 1e-10"
            % (L, W["beta"], m0 if m0 is not None else mass_for(L, W["beta"], W["seed"]), nlev, W["ntv"], W["d"],
               W["k"], W["nrhs_max"], W["eps"]))


# ------------------------------------------------------------------ profiling cases (ncu captures)
def profile_case(args):
    """Small self-contained GPU cases whose kernels an ncu capture can select (-k, -s, -c): the workload's
    hierarchy and one solve on a level, the fine stencil alone, the coarse tensor-core stencil alone, or the
    learned preconditioner's forward.  Prints nothing timed."""
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2303_11512_gb300 import api
    from synthetic import gauge
    W = dict(WORKLOAD)
    if args.tensor_cores is not None:
        W["tensor_cores"] = args.tensor_cores
    L = args.L
    m0 = mass_for(L, W["beta"], W["seed"])
    U = torch.from_numpy(gauge.links(gauge.field(L, W["beta"], W["seed"]))).cuda()
    ctx = api.Context()
    if args.profile_case == "nn":
        # five forward applications of the learned preconditioner (4 layers, 16 channels, tensor-core layers,
        # seeded initial weights) to --profile-nrhs fine-level vectors
        net = api.Net(ctx, U, L, 4, 16, seed=2, tensor_cores=True)
        r = torch.randn((args.profile_nrhs, 2 * L * L), dtype=torch.complex64, device="cuda")
        y = torch.empty_like(r)
        for _ in range(5):
            net.forward(r, y)
        torch.cuda.synchronize()
        net.close()
    elif args.profile_case == "stencil":
        n = 2 * L * L
        x = torch.randn((args.profile_nrhs, n), dtype=torch.complex64, device="cuda")
        y = torch.empty_like(x)
        for _ in range(10):
            api.schwinger_apply(ctx, U, L, m0, x, y, api.FP32)
    else:
        h = api.mg_setup(ctx, U, L, m0, ntv=W["ntv"], bootstrap=args.profile_bootstrap,
                         bootstrap_its=W["bootstrap_its"], pre_smooth=W["pre_smooth"], post_smooth=W["post_smooth"],
                         tensor_cores=W["tensor_cores"])
        lv = args.profile_level
        if args.profile_case == "smooth":
            # ten tensor-core SAP sweeps on level lv (block stencil residuals and block-inverse updates)
            prec = {1: api.BF16, 3: api.FP16}.get(W["tensor_cores"], api.TF32)
            f = torch.randn((args.profile_nrhs, h.n[lv]), dtype=torch.complex64, device="cuda")
            x = torch.zeros_like(f)
            h.smooth(lv, f, x, prec, 10)
            ns = h.side[lv] ** 2
            print("sites", ns, "blocks per colour", ns // 8)
        elif args.profile_case == "coarse":
            # ten tensor-core stencil applications y = D_l x on level lv (no additive input, every rhs active)
            prec = {1: api.BF16, 3: api.FP16}.get(W["tensor_cores"], api.TF32)
            x = torch.randn((args.profile_nrhs, h.n[lv]), dtype=torch.complex64, device="cuda")
            y = torch.empty_like(x)
            for _ in range(10):
                h.apply(lv, x, y, prec)
            ns = h.side[lv] ** 2
            wbytes = ns * 5 * 16 * 32 * (2 if W["tensor_cores"] in (1, 3) else 4)
            print("algorithmic bytes per launch", ns * 256 * args.profile_nrhs + wbytes, "sites", ns)
        else:
            b = api.mgmlmc_rademacher(ctx, 1, 0, 0, 0, h.n[lv], args.profile_nrhs)
            x = torch.empty_like(b)
            st = api.fgmres_batched(ctx, h, lv, b, x, prec=api.MIXED, tol=1e-10)
            print("iters", st["iters"], "relres", st["max_relres"])
        h.close()
    torch.cuda.synchronize()
    ctx.close()
    return 0


def config_records(args):
    """Records of the small configurations: plain Hutchinson (Algorithm 1, unpreconditioned GMRES(30) to 1e-10)
    at L = 16 against the exact trace from the library's dense inverse of D, and MG-MLMC at L = 128 (3 levels, 64
    rhs per launch) in the FP64 and the FP32 / FP64-refinement form.  Times with CUDA events after one untimed
    run; one JSON line."""
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2303_11512_gb300 import api
    from synthetic import gauge
    ctx = api.Context()
    stream = ctx.stream

    def timed(fn, reps=3):
        fn()
        ts, out = [], None
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b) / 1e3)
        return sorted(ts)[len(ts) // 2], out

    # C0: L = 16, beta 3, m0 -0.05, Rademacher, at most 1000 samples
    L0, m00 = 16, -0.05
    U0 = torch.from_numpy(gauge.links(gauge.field(L0, 3.0, 0))).cuda()
    n0 = 2 * L0 * L0
    I = torch.eye(n0, dtype=torch.complex128, device="cuda")
    Dm = torch.empty_like(I)
    api.schwinger_apply(ctx, U0, L0, m00, I, Dm, api.FP64)      # rows = D e_j, i.e. D^T
    Dinv = Dm.transpose(0, 1).contiguous()
    api.mg_dense_inverse(ctx, Dinv, api.FP64)
    exact = complex(torch.diagonal(Dinv).sum().item())
    h0 = api.mg_setup(ctx, U0, L0, m00, ntv=4, setup_sweeps=2)
    t0, r0 = timed(lambda: api.hutchinson_estimate(ctx, h0, eps=0.02, seed=4, precond=0, m=30, tol=1e-10,
                                                   maxit=20000, prec=api.FP64, max_samples=1000))
    h0.close()
    c0 = dict(L=16, time_to_eps_s=t0, eps=0.02, N=r0["N"], tau=[r0["tau"].real, r0["tau"].imag], sigma=r0["sigma"],
              exact=[exact.real, exact.imag], deviation_in_sigma=abs(r0["tau"] - exact) / r0["sigma"])
    # C1: L = 128, beta 3, tuned m0, MG-MLMC (d = 0), 64 rhs per launch, FP64 vs mixed
    L1 = 128
    m01 = mass_for(L1, 3.0, 0)
    U1 = torch.from_numpy(gauge.links(gauge.field(L1, 3.0, 0))).cuda()
    c1 = dict(L=128, m0=m01, eps=1e-3)
    for name, prec in (("fp64", api.FP64), ("mixed", api.MIXED)):
        def run():
            h = api.mg_setup(ctx, U1, L1, m01, ntv=8)
            r = api.trace_estimate(ctx, h, eps=1e-3, d=0, k=1, nrhs_max=64, nrhs_first=16, cost_mode=1, seed=3,
                                   prec=prec)
            h.close()
            return r
        t, r = timed(run)
        c1[name] = dict(time_to_eps_s=t, N=r["N"], solves=r["solves"], tau=[r["tau"].real, r["tau"].imag],
                        rel_sigma=r["sigma"] / abs(r["tau"]))
    c1["speedup_mixed_vs_fp64"] = c1["fp64"]["time_to_eps_s"] / c1["mixed"]["time_to_eps_s"]
    print(json.dumps({"record": "configs", "hutchinson_L16": c0, "mlmc_L128": c1}), flush=True)
    ctx.close()
    return 0


def ensemble_record(args):
    """Ensemble record: time to eps of every field (set-up included) and the whole-ensemble throughput."""
    import __graft_entry__ as g
    g.build()
    from paper_2303_11512_gb300 import ensemble
    out = ensemble.run_c4(n=16, eps=args.eps, concurrency=args.ensemble, workload=WORKLOAD)
    fields = [dict(name=r["name"], L=r["L"], m0=r["m0"], N=r["N"], solves=r["solves"],
                   setup_s=round(r["setup_s"], 4), time_to_eps_s=round(r["time_s"], 4),
                   rel_sigma=r["sigma"] / abs(complex(*r["tau"]))) for r in out["runs"]]
    print(json.dumps({"metric": "ensemble_wall_time_to_eps", "value": out["wall_s"], "unit": "s",
                      "higher_is_better": False, "eps": args.eps, "concurrency": args.ensemble,
                      "fields_per_s": out["fields_per_s"], "solves_per_s": out["solves_per_s"],
                      "admitted": len(out["runs"]), "rejected": out["rejected"], "groups": out["groups"],
                      "data": "synthetic quenched U(1), beta 3", "fields": fields}), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=WORKLOAD["L"])
    ap.add_argument("--eps", type=float, default=WORKLOAD["eps"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparator run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end pass")
    ap.add_argument("--timing-filter", default="")
    ap.add_argument("--tensor-cores", type=int, default=None, choices=[0, 1, 2, 3],
                    help="coarse-level tensor-core operands: 1 BF16, 2 TF32, 3 FP16, 0 CUDA cores (default: the workload's)")
    ap.add_argument("--profile-case", choices=["solve", "stencil", "coarse", "smooth", "nn"], default=None,
                    help="run one small case for an ncu capture instead of the benchmark: 'solve' = one mixed "
                         "FGMRES solve on --profile-level with --profile-nrhs rhs on the workload hierarchy, "
                         "'stencil' = ten FP32 fine-stencil applications to --profile-nrhs vectors, 'coarse' = ten "
                         "tensor-core stencil applications on --profile-level, 'smooth' = ten tensor-core SAP sweeps "
                         "on --profile-level, 'nn' = five forward applications of the learned preconditioner")
    ap.add_argument("--profile-level", type=int, default=1)
    ap.add_argument("--profile-nrhs", type=int, default=64)
    ap.add_argument("--profile-bootstrap", type=int, default=WORKLOAD["bootstrap"],
                    help="bootstrap rounds of the profiled hierarchy (0: no tensor-core launches before the solve)")
    ap.add_argument("--configs", action="store_true",
                    help="instead of the benchmark, print the records of the L = 16 plain Hutchinson and the L = 128 "
                         "MG-MLMC (FP64 vs mixed) configurations")
    ap.add_argument("--ensemble", type=int, default=0, metavar="CONCURRENCY",
                    help="instead of the benchmark, run the 16-field ensemble (L 128..1024, three masses) with up "
                         "to CONCURRENCY fields at a time and print its record as one JSON line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return profile_case(args)
    if args.ensemble:
        return ensemble_record(args)
    if args.configs:
        return config_records(args)

    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    import __graft_entry__ as g
    g.build()
    from paper_2303_11512_gb300 import api
    from paper_2303_11512_gb300.estimator import TraceEstimator
    from synthetic import gauge

    W = dict(WORKLOAD)
    W["L"], W["eps"] = args.L, args.eps
    if args.tensor_cores is not None:
        W["tensor_cores"] = args.tensor_cores
    L = W["L"]
    seed = replica_seed(W["seed"], rank)
    m0 = mass_for(L, W["beta"], W["seed"])
    U_host = gauge.links(gauge.field(L, W["beta"], seed))
    U = torch.from_numpy(U_host).cuda()
    mgp = dict(ntv=W["ntv"], bootstrap=W["bootstrap"], bootstrap_its=W["bootstrap_its"],
               kcycle_its=W["kcycle_its"], pre_smooth=W["pre_smooth"], post_smooth=W["post_smooth"],
               tensor_cores=W["tensor_cores"], autotune=W["autotune"])
    estp = dict(eps=W["eps"], d=W["d"], k=W["k"], nrhs_max=W["nrhs_max"], nrhs_first=W["nrhs_first"], cost_mode=1,
                seed=0)
    stream = torch.cuda.current_stream()
    ctx = api.Context(stream)

    def step(prec=api.MIXED, **over):
        h = api.mg_setup(ctx, U, L, m0, **mgp)
        r = api.trace_estimate(ctx, h, prec=prec, **dict(estp, **over))
        h.close()
        return r

    for _ in range(args.warmup):
        res = step()
    # timed region: device-resident field, CUDA events on the library's stream
    clocks = ClockSampler(local)
    ctx.timing(True, args.timing_filter or None)
    launches0 = ctx.launches
    barrier()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    results = [step() for _ in range(args.steps)]
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ctx.timing(False)
    launches = ctx.launches - launches0
    ms = e0.elapsed_time(e1) / args.steps
    rpt = ctx.timing_report()
    ms = max_over_ranks(ms, world)
    value = ms / 1e3

    # dominant kernel -> roofline (CUDA-core FMA peaks measured on this GPU by the library)
    P = peaks()
    P["fp64_alu_tflops"] = api.alu_peak(ctx, True)
    P["fp32_alu_tflops"] = api.alu_peak(ctx, False)
    dom, info = max(rpt.items(), key=lambda kv: kv[1]["ms"])
    tot_ms = sum(v["ms"] for v in rpt.values())
    avg_ms = info["ms"] / info["launches"]
    bytes_l = info["bytes"] / info["launches"]
    flops_l = info["flops"] / info["launches"]
    ai = flops_l / max(bytes_l, 1.0)
    fp64 = "double" in dom
    tensor = dom.startswith("k_tc")  # TF32 tcgen05 kernels: compute roof is the TF32 tensor rate
    if tensor:
        comp_peak, comp_bound = P["tf32_tensor_tflops_sustained"], "tensor"
    else:
        comp_peak, comp_bound = (P["fp64_alu_tflops"] if fp64 else P["fp32_alu_tflops"]), "alu"
    ridge = comp_peak * 1e12 / (P["hbm_gbs"] * 1e9)
    if ai <= ridge:
        roof = dict(bound="hbm", achieved=bytes_l / (avg_ms * 1e-3) / 1e9, peak=P["hbm_gbs"], unit="GB/s")
    else:
        roof = dict(bound=comp_bound, achieved=flops_l / (avg_ms * 1e-3) / 1e12, peak=comp_peak, unit="TFLOP/s")
    roof["frac"] = roof["achieved"] / roof["peak"]
    # DRAM traffic of the dominant kernel: the ncu capture of one launch (dram__bytes_read + _write) relative to
    # that launch's algorithmic bytes, scaled to this run's average launch (the bench's launches mix levels and
    # batch sizes; the captures are level-1, 32-rhs launches, TRAFFIC_PER_ALG_BYTE)
    traffic, traffic_src = None, None
    for key, (ratio, src) in TRAFFIC_PER_ALG_BYTE.items():
        if key in dom:
            traffic, traffic_src = ratio * bytes_l, src
    roof.update(kernel=dom, launches=info["launches"], avg_launch_ms=avg_ms, share=info["ms"] / max(tot_ms, 1e-9),
                bytes_per_launch=bytes_l, flops_per_launch=flops_l, peak_src=P["src"], traffic=traffic,
                traffic_src=traffic_src)
    kernels = {k: dict(launches=v["launches"], ms=round(v["ms"], 3), share=round(v["ms"] / max(tot_ms, 1e-9), 4),
                       gbs=round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1),
                       tflops=round(v["flops"] / max(v["ms"], 1e-9) / 1e9, 3))
               for k, v in sorted(rpt.items(), key=lambda kv: -kv[1]["ms"])[:12]}

    # fine stencil alone in the workload's launch shape (FP32, 256 rhs): HBM GB/s
    n = 2 * L * L
    xs = torch.randn((W["nrhs_max"], n), dtype=torch.complex64, device="cuda")
    ys = torch.empty_like(xs)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        api.schwinger_apply(ctx, U, L, m0, xs, ys, api.FP32)
    ts = []
    for _ in range(10):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        api.schwinger_apply(ctx, U, L, m0, xs, ys, api.FP32)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ts.sort()
    st_bytes = W["nrhs_max"] * L * L * 32 + L * L * 16
    stencil = dict(gbs=st_bytes / (ts[len(ts) // 2] * 1e-3) / 1e9, ms=ts[len(ts) // 2], nrhs=W["nrhs_max"],
                   frac_hbm=st_bytes / (ts[len(ts) // 2] * 1e-3) / 1e9 / P["hbm_gbs"])
    del xs, ys, flush

    # end to end through the public API: host gauge field, H2D + set-up + estimate + result D2H
    e2e = None
    if not args.no_e2e:
        U_pin = torch.from_numpy(U_host).pin_memory()
        barrier()
        e2e_t = []
        for _ in range(max(1, args.steps)):
            t1 = time.perf_counter()
            est = TraceEstimator(U_pin.numpy(), L, m0, ctx=ctx, pinned=False, **mgp)
            est.run(**estp)
            est.close()
            torch.cuda.synchronize()
            e2e_t.append(time.perf_counter() - t1)
        e2e = dict(value=sum(e2e_t) / len(e2e_t), unit="s", h2d_bytes_per_step=int(U_host.nbytes),
                   d2h_bytes_per_step=int(16 * 2))

    # the same time to eps with a smaller sketch (d = 16, k = 1: 32 difference-operator applications per level),
    # median of three after one untimed run
    alt_runs = []
    barrier()
    step(d=16, k=1)
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ra = step(d=16, k=1)
        b.record(stream)
        torch.cuda.synchronize()
        alt_runs.append(a.elapsed_time(b) / 1e3)
    sketch_alt = dict(d=16, k=1, time_to_eps_s=sorted(alt_runs)[1], runs_s=alt_runs, N=ra["N"], solves=ra["solves"],
                      rel_sigma=ra["sigma"] / abs(ra["tau"]))

    # plain FP64 batched MG form of the same estimator (the comparator of the metric): one untimed run, then the
    # median of three
    fp64_s, fp64_runs = None, []
    if not args.no_fp64:
        barrier()
        step(api.FP64)
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(api.FP64)
            b.record(stream)
            torch.cuda.synchronize()
            fp64_runs.append(a.elapsed_time(b) / 1e3)
        fp64_s = sorted(fp64_runs)[1]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count()))
        orc = OracleWorkload(U_host, L, m0, W["seed"])
        orc.batch(4)
        Nl = results[-1]["N"]
        cpu = dict(value=orc.total(Nl, W["d"], W["k"]), unit="s", cores=os.cpu_count(), kind="oracle",
                   sample=orc.describe(Nl, W["d"], W["k"], 4) + " (N_l: this run's)")

    r = results[-1]
    if rank == 0:
        line = dict(
            metric="time_to_eps_s", value=value, unit="s", n_gpus=world, steps=args.steps, warmup=args.warmup,
            ms_per_step=ms, higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f32+f64",
            data="synthetic",
            config=dict(workload=workload_name(W, L, m0, len(r["N"]) + 1),
                        l2="inputs larger than L2 (fine vectors 0.5-2 GB per batch); stencil timing flushes L2",
                        bootstrap=W["bootstrap"], kcycle_its=W["kcycle_its"],
                        vcycle="V(%d,%d) SAP" % (W["pre_smooth"], W["post_smooth"])),
            roofline=roof, cpu_baseline=cpu, e2e=e2e, gpu_launches=int(launches),
            clocks=clk, fp64_reference_s=fp64_s, fp64_reference_runs_s=fp64_runs,
            speedup_vs_fp64=(fp64_s / value) if fp64_s else None,
            sketch_d16_k1=sketch_alt,
            alu_peaks=dict(fp64_tflops=P["fp64_alu_tflops"], fp32_tflops=P["fp32_alu_tflops"],
                           src="measured: mgmlmc_alu_peak (8 FMA chains per thread, full grid)"),
            stencil_fp32=stencil,
            estimate=dict(tau=[r["tau"].real, r["tau"].imag], sigma=r["sigma"], rel_sigma=r["sigma"] / abs(r["tau"]),
                          N=r["N"], computed=r["computed"], solves=r["solves"], inner_iters=r["inner_iters"]),
            kernels=kernels,
            tuning=[[api.TUNE_KINDS.get(e["kind"], e["kind"]), e["side"], e["bucket"], e["format"], e["variant"],
                     round(e["us"], 1)] for e in api.tune_table()])
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
