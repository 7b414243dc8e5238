"""Benchmark: semi-implicit spectral Cahn-Hilliard steps at 1024^3 on GB300.

One bench step = one time step of the scheme (all four passes) over the
1024^3 field (c0 = 0.3 + U(-0.05, 0.05), seed 0, dt = 0.1, M = kappa = 1,
h = 1; 200 steps by default). Prints one JSON line (rank 0).

  value      voxel-steps/s of the K timed steps, inputs resident in HBM
  e2e        the same metric for the whole job through the host API:
             host c0 (pinned) -> evx_set_field_host -> K steps -> evx_get_field_host
  roofline   dominant kernel: algorithmic bytes / CUDA-event duration (same timed region)
  cpu_baseline  the FP64 oracle timed on the host cores on a bounded sample

--impl reference times the FP64 oracle (the CPU reference of this method) on
the host cores for the same metric.
With torchrun (N > 1) each rank runs an independent replica of the job (the
method has no data-parallel exchange for one field); value = all ranks'
voxel-steps / max time over ranks.
"""
import argparse
import json

import numpy as np
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CH voxel-steps/s at 1024^3"
UNIT = "voxel-steps/s"
DT, MOB, KAPPA, H = 0.1, 1.0, 1.0, 1.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="evx", choices=["evx", "reference"])
    ap.add_argument("--n", type=int, default=1024, help="grid edge (default 1024)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-small", action="store_true", help="skip the 64^3 / 256^3 / 400^3 timings")
    ap.add_argument("--no-design-b", action="store_true", help="skip the fused-pass (5-sweep) timing")
    ap.add_argument("--train-iters", type=int, default=1500)
    ap.add_argument("--ac-steps", type=int, default=50, help="Allen-Cahn steps timed after the CH run (0: skip)")
    ap.add_argument("--vm-steps", type=int, default=20,
                    help="variable-mobility CH steps timed after the CH run (0: skip)")
    ap.add_argument("--step-probe", default=None, metavar="NX,NY,NZ,STEPS",
                    help="only run STEPS Cahn-Hilliard steps on an NX x NY x NZ grid and exit (for profilers)")
    ap.add_argument("--conv-probe", default=None, metavar="B,X,Y,Z[,EPI]",
                    help="only time the surrogate's 32->32 convolution (plain epilogue) on this shape and exit")
    return ap.parse_args()


def max_over_ranks(x: float) -> float:
    """Largest x over the ranks of the default process group (x itself when not
    distributed). NCCL groups reduce a CUDA tensor, others a CPU tensor."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world_size: int, steps: int, voxels: float, seconds: float) -> float:
    """Whole-job voxel-steps/s: every rank advances its own replica of the field
    (weak scaling), timed by the slowest rank."""
    return world_size * steps * voxels / seconds


def replica_seed(rank: int) -> int:
    """Seed of the initial field of replica ``rank`` (independent trajectories)."""
    return rank


def kernel_source(text, names):
    """The definitions of the named functions in a C++ source (signature line
    through the matching closing brace), concatenated: the part of a file a
    kernel's memory traffic depends on."""
    out = []
    for name in names:
        i = text.find(" " + name + "(")
        if i < 0:
            return None
        i = text.rfind("\n", 0, text.rfind("template", 0, i) if "template" in text[max(0, i - 200):i] else i) + 1
        j = text.index("{", text.index(name + "(", i))
        depth = 0
        for k in range(j, len(text)):
            depth += {"{": 1, "}": -1}.get(text[k], 0)
            if depth == 0:
                out.append(text[i:k + 1])
                break
    return "\n".join(out)


def measured_traffic(dominant_pass: int, alg_bytes: float):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary (profiles/traffic_x_pass.json: traffic / algorithmic bytes on a
    smaller case), or None when that kernel's source (its definition, its
    launcher and the tensor-map builder) has changed since."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic_x_pass.json")) as f:
            d = json.load(f)
        with open(os.path.join(ROOT, d["source"])) as f:
            src = kernel_source(f.read(), d["functions"])
        sha = hashlib.sha256(src.encode()).hexdigest() if src else None
    except Exception:
        return None
    if dominant_pass != 0 or sha is None or sha != d.get("functions_sha256"):
        return None
    return d["traffic_over_algorithmic"] * alg_bytes


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling every 20 ms from before the warm-up steps to after the
    timed region; the record reports the samples taken inside the timed region
    (host wall-clock bracket) and, for context, all samples under load."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, t0=None, t1=None):
        """t0, t1: time.time() bracket of the timed region (samples inside it are
        the record; a sample is attributed to the 20 ms before its timestamp)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        import datetime
        rows, mx = [], None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                sm = float(f[2])
                mx = float(f[3])
                pw = float(f[4])
            except ValueError:
                continue
            rows.append((ts, sm, pw, {nm for nm, v in zip(names, f[6:10]) if v.lower() == "active"}))
        os.unlink(self.path)
        inside = [r for r in rows if t0 is not None and t0 <= r[0] <= t1 + 0.02]
        loaded = [r for r in rows if r[2] > 300.0]  # under load (power draw above idle)

        def med(xs):
            xs = sorted(xs)
            return xs[len(xs) // 2] if xs else None

        rec = inside if inside else loaded
        reasons = set()
        for r in rec:
            reasons |= r[3]
        return {"sm_mhz": med([r[1] for r in rec]), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(inside), "interval_ms": 20,
                "run_sm_mhz": med([r[1] for r in loaded]), "run_samples_under_load": len(loaded),
                "run_reasons": sorted(set().union(*[r[3] for r in loaded])) if loaded else []}


def cpu_baseline_oracle(n_sample=256, steps=2):
    """FP64 oracle step on an n_sample^3 grid with the same recipe; voxel-steps/s."""
    from oracle import oracle as O
    from paper_2507_21748_gb300 import inputs
    c0 = inputs.uniform_field((n_sample,) * 3, seed=0, offset=0.3)
    O.ch_step(c0[:8, :8, :8], DT, MOB, KAPPA, H, 1)  # load / warm the library
    t0 = time.perf_counter()
    O.ch_step(c0, DT, MOB, KAPPA, H, steps, check_imag=False)
    dt = time.perf_counter() - t0
    return {"value": steps * n_sample ** 3 / dt, "unit": UNIT, "cores": O.num_threads(),
            "kind": "oracle",
            "sample": "FP64 oracle (full complex 3D FFT, numpy + C/OpenMP), %d steps of the same "
                      "recipe on a %d^3 grid (%.1f s); its per-voxel cost grows with log V, so "
                      "at 1024^3 it would be no faster" % (steps, n_sample, dt)}


def cpu_single_thread_oracle(n_sample=128, steps=1):
    """The same oracle step on one host core (OMP_NUM_THREADS=1 in a child process,
    since the OpenMP runtime reads it once at load)."""
    code = ("import sys, time, json; sys.path.insert(0, %r)\n"
            "from oracle import oracle as O\n"
            "from paper_2507_21748_gb300 import inputs\n"
            "c0 = inputs.uniform_field((%d,) * 3, seed=0, offset=0.3)\n"
            "O.ch_step(c0[:8, :8, :8], %r, %r, %r, %r, 1)\n"
            "t0 = time.perf_counter(); O.ch_step(c0, %r, %r, %r, %r, %d, check_imag=False)\n"
            "print(json.dumps({'s': time.perf_counter() - t0, 'threads': O.num_threads()}))\n"
            ) % (ROOT, n_sample, DT, MOB, KAPPA, H, DT, MOB, KAPPA, H, steps)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": steps * n_sample ** 3 / d["s"], "unit": UNIT, "cores": d["threads"], "kind": "oracle",
            "sample": "same oracle, one thread, %d step(s) on a %d^3 grid (%.1f s)" % (steps, n_sample, d["s"])}


def sampled_modes(n, count=14, seed=1):
    """Wave vectors for the sampled-mode checks: fixed low, Nyquist and fastest-
    growing modes plus random ones (k = 0 excluded; it is reported on its own)."""
    rng = np.random.default_rng(seed)
    fixed = np.array([[1, 0, 0], [0, 0, 1], [0, 0, n // 2], [n // 2, n // 2, n // 2], [114 * n // 1024, 0, 0],
                      [3, 5, 7]])
    return np.concatenate([fixed, rng.integers(0, n, size=(count - len(fixed), 3))])


def mode_error(got_modes, want_modes, field_l2):
    """Sampled-mode errors: the maximum |delta c_hat(k)| over the modes and the
    estimate of the whole-field relative L2 it implies (by Parseval, the field's
    rel. L2 error is the RMS of |delta c_hat| over all modes over ||c||_2)."""
    d = np.abs(np.asarray(got_modes) - np.asarray(want_modes))
    return {"modes": len(d), "max_abs_mode_err": float(d.max()),
            "rel_l2_estimate": float(np.sqrt(np.mean(d * d)) / field_l2)}


def field_l2(c):
    return float(np.sqrt(sum(float(np.sum(np.asarray(c[i:i + 64], dtype=np.float64) ** 2))
                             for i in range(0, c.shape[0], 64))))


def bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def adjoint_bench(n=128, nsteps=200, ckpt=20):
    """The differentiable inverse run's cost: one gradient (adjoint of nsteps steps with
    checkpoints every ckpt steps, forward recomputation included) against the forward
    run alone, at n^3 with kappa = 1.5, M = 0.8 (the target configuration's parameters).
    The gradient is checked against the FP64 oracle's adjoint on a 32^3 sample of the
    same recipe (outside the timing)."""
    import torch
    from oracle import oracle as O
    from paper_2507_21748_gb300 import evx, inputs
    shape = (n, n, n)
    c0 = torch.from_numpy(inputs.uniform_field(shape, seed=0)).cuda()
    dL = torch.from_numpy(inputs.uniform_field(shape, seed=5, lo=-1.0, hi=1.0)).cuda()
    g = evx.Grid(shape, dt=DT, M=0.8, kappa=1.5, h=H)
    g.set_field(c0)
    g.step(nsteps)  # builds the step graphs
    g.adjoint(c0, nsteps, ckpt, dL)  # allocates the segment store
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g.set_field(c0)
    g.step(nsteps)
    out = g.get_field()
    e1.record()
    torch.cuda.synchronize()
    t_fwd = e0.elapsed_time(e1)
    t0 = time.perf_counter()
    g0, gk, gm = g.adjoint(c0, nsteps, ckpt, dL)  # synchronises
    t_adj = 1e3 * (time.perf_counter() - t0)
    del out, g0
    g.close()
    # accuracy against the FP64 oracle adjoint (small sample of the same recipe)
    m = 32
    cs = inputs.uniform_field((m,) * 3, seed=0)
    ds = inputs.uniform_field((m,) * 3, seed=5, lo=-1.0, hi=1.0)
    gs = evx.Grid((m,) * 3, dt=DT, M=0.8, kappa=1.5, h=H)
    a0, ak, am = gs.adjoint(torch.from_numpy(cs).cuda(), 40, ckpt, torch.from_numpy(ds).cuda())
    gs.close()
    r0, rk, rm = O.ch_adjoint(cs, ds, DT, 0.8, 1.5, H, 40)
    a0 = a0.cpu().numpy()
    return {"workload": "%d^3, %d steps, checkpoint every %d, kappa = 1.5, M = 0.8, dL/dc_N = U(-1, 1)"
                        % (n, nsteps, ckpt),
            "forward_ms": t_fwd, "gradient_ms": t_adj, "gradient_over_forward": t_adj / t_fwd,
            "error_vs_oracle": {"what": "32^3, 40 steps, same recipe: FP32 GPU adjoint vs FP64 oracle adjoint",
                                "dLdc0_rel_l2": float(np.linalg.norm(a0 - r0) / np.linalg.norm(r0)),
                                "dLdkappa_rel": abs(ak - rk) / abs(rk), "dLdM_rel": abs(am - rm) / abs(rm)}}


def surrogate_bench(args):
    """Learned surrogate (10 solver steps per block): the CNN corrects the block
    propagator (the scheme's linear part exact over the block, its nonlinear
    remainder frozen; one step's cost). Train at 128^3 on solver trajectories
    (seeds 0..255, mean in [-0.3, 0.3], noise 0.05, 300 steps each), then advance
    8 fields of 256^3 by 30 blocks (300 steps: noise decay, spinodal growth and
    the start of coarsening) with the guarded surrogate, the propagator alone and
    the plain solver; report times, errors against the solver and the conv
    kernel's tensor throughput."""
    import torch
    from paper_2507_21748_gb300 import evx, inputs
    from paper_2507_21748_gb300 import surrogate as S
    out = {}
    tr_shape, B = (128, 128, 128), 4
    pool = S.TrajectoryPool(tr_shape, B, block=10, horizon=300, seeds=range(256), base=True)
    net = S.Net(tr_shape, B, seed=0, proj_gain=1e-3)  # FP32 residual stream (default)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = S.train(net, pool, args.train_iters, lr=5e-4, lr_final=1e-4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    out["train"] = {"grid": "128^3", "batch": B, "iters": args.train_iters, "pairs": B * args.train_iters,
                    "trajectories": min(256, pool.next_seed), "horizon_steps": 300, "seconds": t_train,
                    "target": "c_{n+10} - block propagator(c_n)",
                    "loss_first": hist[0], "loss_last": float(np.mean(hist[-10:]))}
    pool.close()
    shape, NB = (256, 256, 256), 8
    inf = S.Net(shape, NB, train=False)
    inf.load_params(net)
    del net
    seeds = range(1000, 1000 + NB)
    c0 = torch.stack([torch.from_numpy(inputs.uniform_field(shape, seed=s, offset=inputs.trajectory_mean(s)))
                      for s in seeds]).cuda()
    out["inference"] = []
    for blocks in (15, 30):
        # plain solver: 8 fields x 10 blocks steps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ref = S.solver_run(c0, 10 * blocks)
        torch.cuda.synchronize()
        t_solver = time.perf_counter() - t0
        # block propagator alone (the method without the network)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bro = S.base_rollout(c0, blocks)
        torch.cuda.synchronize()
        t_base = time.perf_counter() - t0
        # surrogate (propagator + network) + guards + fallback
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got, st = S.rollout(inf, c0, blocks, base=True)
        torch.cuda.synchronize()
        t_sur = time.perf_counter() - t0
        r = ref.double().flatten(1)

        def relmax(x):
            return float(((x.double() - ref.double()).flatten(1).norm(dim=1) / r.norm(dim=1)).max())

        rel, rel_base, persist = relmax(got), relmax(bro), relmax(c0)
        out["inference"].append({
            "grid": "256^3", "batch": NB, "blocks_per_field": blocks, "steps_per_block": 10,
            "t_solver_s": t_solver, "t_surrogate_path_s": t_sur,
            "speedup_vs_solver": t_solver / t_sur, "rel_l2_vs_solver_max": rel, "meets_1e-2": rel <= 1e-2,
            "without_network": {"what": "block propagator alone (evx_ch_block), same blocks, no guard",
                                "t_s": t_base, "speedup_vs_solver": t_solver / t_base,
                                "rel_l2_vs_solver_max": rel_base, "meets_1e-2": rel_base <= 1e-2},
            "network_gain": rel_base / rel if rel > 0 else None,
            "rel_l2_persistence_max": persist,
            "block_evaluations": st["blocks"], "fallbacks": st["fallbacks"],
            "t_net_s": st["t_net_s"], "t_base_s": st["t_base_s"], "t_guard_s": st["t_guard_s"],
            "t_fallback_s": st["t_fallback_s"]})
        del ref, bro, got
    # conv 32 -> 32 throughput at 256^3 x 8 (dominant surrogate kernel), both engines
    X, Y, Z = shape
    flops = 2.0 * 27 * 32 * 32 * NB * X * Y * Z
    peak, src = bf16_peak()

    def conv_ms(engine):
        S.set_conv_engine(engine)
        try:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            for _ in range(2):
                inf._conv(inf.h[0], "W1_0", inf.p["b1_0"], inf.a[0], 32, 32, S.EPI_GELU, pre=inf.u[0])
            e0.record()
            reps = 5
            for _ in range(reps):
                inf._conv(inf.h[0], "W1_0", inf.p["b1_0"], inf.a[0], 32, 32, S.EPI_GELU, pre=inf.u[0])
            e1.record()
            S.check()
            return e0.elapsed_time(e1) / reps
        finally:
            S.set_conv_engine(S.ENGINE_TCGEN05)

    ms = conv_ms(S.ENGINE_TCGEN05)
    ms_sync = conv_ms(S.ENGINE_MMA_SYNC)
    out["conv_roofline"] = {"bound": "tensor",
                            "kernel": "conv_ring_kernel<GELU> (tcgen05.mma bf16, TMEM accumulators, TMA ring), "
                                      "as inference runs it: GELU output only, no pre-activation store",
                            "achieved": flops / (ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                            "frac": flops / (ms * 1e-3) / 1e12 / peak, "peak_source": src + " bf16_tflops",
                            "ms_per_launch": ms,
                            "mma_sync_engine": {"kernel": "conv_fwd_kernel<32,32,GELU> (mma.sync bf16)",
                                                "ms_per_launch": ms_sync,
                                                "achieved": flops / (ms_sync * 1e-3) / 1e12}}
    del inf
    torch.cuda.empty_cache()
    return out


def small_grid_bench():
    """The smaller configurations: 64^3 (100-step runs; L2-resident, so latency,
    not bandwidth) and 256^3 / 400^3 (1000-step runs) with the same recipe as the
    parity tests (c0 = U(-0.05, 0.05), seed 0); CUDA-graph launches, CUDA events."""
    import torch
    from oracle import oracle as O
    from paper_2507_21748_gb300 import evx, inputs
    out = {}
    for n, steps in ((64, 1000), (256, 1000), (400, 1000)):
        shape = (n, n, n)
        c0 = inputs.uniform_field(shape, seed=0)
        g = evx.Grid(shape, dt=DT, M=MOB, kappa=KAPPA, h=H)
        # error after one step against the FP64 oracle, whole field (outside the timed region)
        g.set_field(torch.from_numpy(c0).cuda())
        g.step(1)
        c1 = g.get_field().cpu().numpy().astype(np.float64)
        ref = O.ch_step(c0, DT, MOB, KAPPA, H, 1, check_imag=False)
        rel = float(np.linalg.norm(c1 - ref) / np.linalg.norm(ref))
        del c1, ref
        g.set_field(torch.from_numpy(c0).cuda())
        g.step(20)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.step(steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out["%d^3" % n] = {"steps": steps, "us_per_step": 1e3 * ms / steps,
                           "voxel_steps_per_s": steps * float(n) ** 3 / (ms * 1e-3),
                           "footprint_bytes": g.footprint(),
                           "kernels": ("fast, L = 32 x TP" if n in (64, 128, 256, 512, 1024)
                                       else "fast, L = 20 x 20 (x, y), M = 200 = 20 x 10 (z)")
                           + ("; fused y-z-y pass" if g.pass_bytes(2) == 0.0 else ""),
                           "error_vs_oracle": {"rel_l2_one_step": rel, "what": "whole field, one step from "
                                               "c0 = U(-0.05, 0.05) seed 0, FP64 oracle"}}
        g.close()
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return
    from oracle import oracle as O
    from paper_2507_21748_gb300 import inputs
    n = 128
    c = inputs.uniform_field((n,) * 3, seed=0, offset=0.3).astype("float64")
    for _ in range(args.warmup):
        c = O.ch_step(c, DT, MOB, KAPPA, H, 1, check_imag=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        c = O.ch_step(c, DT, MOB, KAPPA, H, 1, check_imag=False)
    dt = time.perf_counter() - t0
    v = args.steps * n ** 3 / dt
    sample = ("FP64 oracle, each step one scheme step of the same recipe on a %d^3 grid "
              "(the 1024^3 field needs ~50 GB of host FP64 arrays per step)" % n)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": "CH 3D periodic, oracle sample %d^3" % n,
                                         "dt": DT, "M": MOB, "kappa": KAPPA},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def conv_probe(spec):
    """Times the surrogate's 32 -> 32 convolution (default engine) on one
    shape, B,X,Y,Z[,EPI] with EPI 0 = plain (default) or 1 = GELU (stores the
    pre-activation too): a small, self-contained case for profilers."""
    import torch
    from paper_2507_21748_gb300 import surrogate as S
    vals = [int(v) for v in spec.split(",")]
    B, X, Y, Z = vals[:4]
    epi = S.EPI_GELU if len(vals) > 4 and vals[4] == 1 else S.EPI_PLAIN
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((B, X, Y, Z, 32), device="cuda", generator=g).to(torch.bfloat16)
    w = (torch.randn((27, 32, 32), device="cuda", generator=g) * 0.1).to(torch.bfloat16)
    b = torch.randn(32, device="cuda", generator=g)
    out = torch.empty_like(x)
    pre = torch.empty_like(x) if epi == S.EPI_GELU else None

    def run():
        S._ck(S.lib.evx_nn_conv3d(S._p(x), S._p(w), S._p(b), S._p(out), S._p(pre) if pre is not None else None,
                                  None, B, X, Y, Z, 32, 32, epi, S._stream()))

    for _ in range(3):
        run()
    S.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        run()
    e1.record()
    S.check()
    ms = e0.elapsed_time(e1) / 5
    flops = 2.0 * 27 * 32 * 32 * B * X * Y * Z
    print(json.dumps({"conv_probe": [B, X, Y, Z], "epilogue": "gelu" if epi == S.EPI_GELU else "plain",
                      "engine": S.conv_engine(), "ms": ms,
                      "tflops": flops / (ms * 1e-3) / 1e12}), flush=True)


def step_probe(spec):
    """Runs a few Cahn-Hilliard steps (same recipe as the bench) on one grid:
    a small, self-contained case for profilers (4 kernels per step after the
    set-field kernels)."""
    import torch
    from paper_2507_21748_gb300 import evx, inputs
    nx, ny, nz, steps = (int(v) for v in spec.split(","))
    c0 = torch.from_numpy(inputs.uniform_field((nx, ny, nz), seed=0, offset=0.3)).cuda()
    g = evx.Grid((nx, ny, nz), dt=DT, M=MOB, kappa=KAPPA, h=H)
    g.set_field(c0)
    g.step(steps)
    torch.cuda.synchronize()
    print(json.dumps({"step_probe": [nx, ny, nz, steps], "mean": g.mean()}), flush=True)
    g.close()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.conv_probe:
        return conv_probe(args.conv_probe)
    if args.step_probe:
        return step_probe(args.step_probe)
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2507_21748_gb300 import evx, inputs

    n = args.n
    shape = (n, n, n)
    V = float(n) ** 3
    c0 = inputs.uniform_field(shape, seed=replica_seed(rank), offset=0.3)
    c0_dev = torch.from_numpy(c0).cuda()
    stream = torch.cuda.current_stream()
    g = evx.Grid(shape, dt=DT, M=MOB, kappa=KAPPA, h=H, stream=stream)
    clocks = Clocks(local)
    clocks.start()
    g.set_field(c0_dev)
    g.step(max(args.warmup, 0))
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # ---- device-resident timed region (per-pass CUDA events on the grid's stream)
    g.set_profiling(True)
    g.pass_times(reset=True)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    w0 = time.time()
    e0.record(stream)
    g.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    w1 = time.time()
    barrier()
    time.sleep(0.05)  # one more sample after the region
    clk = clocks.stop(w0, w1)
    ms = e0.elapsed_time(e1)
    pass_ms, pass_cnt = g.pass_times(reset=True)
    g.set_profiling(False)
    t_max = max_over_ranks(ms)
    value = job_throughput(ws, args.steps, V, t_max * 1e-3)

    # roofline of the dominant pass
    fused = g.pass_bytes(2) == 0.0  # the y inverse, z step and y forward run as one fused pass
    names = ["x pass + k-space update", "y inverse", "z C2R + c^3-c + R2C", "y forward"]
    if fused:
        names = ["x pass + k-space update", "fused y inverse + z C2R/c^3-c/R2C + y forward (x slabs in L2)",
                 "(in the fused pass)", "(in the fused pass)"]
    fast = n in (64, 128, 256, 512, 1024, 400) and os.environ.get("EVX_GENERIC", "") != "1"
    r1, tp = (20, 20) if n == 400 else (32, max(n // 32, 2))  # four-step split n = R1 x TP
    rz, tz, ntz = (20, 10, 160) if n == 400 else (32, max(tp // 2, 2), 128)  # z pass: M = n / 2
    kern = (["fast::fxupd_tma_kernel<%d, %d>" % (r1, tp), "fast::fspass_tma_kernel<%d, %d, 1>" % (r1, tp),
             "fast::fzstep_kernel<%d, %d, %d>" % (rz, tz, ntz), "fast::fspass_tma_kernel<%d, %d, -1>" % (r1, tp)]
            if fast else ["xupdate_kernel", "spass_kernel<1>", "zpass_kernel<Z_STEP>", "spass_kernel<-1>"])
    if fused:
        kern[1] = "fused::fyzy_kernel<%d, %d, %d, %d>" % (r1, tp, rz, tz)
        kern[2] = kern[3] = "-"
    dom = max(range(4), key=lambda k: pass_ms[k])
    avg_ms = pass_ms[dom] / max(pass_cnt[dom], 1)
    alg_bytes = g.pass_bytes(dom)
    peak, peak_src = peaks()
    achieved = alg_bytes / (avg_ms * 1e-3) / 1e9
    step_bytes = sum(g.pass_bytes(k) for k in range(4))
    field_bytes = g.pass_bytes(0) / 3.0  # F: one half-spectrum field, nx ny (nz/2 + 1) complex64
    per_pass = {}
    for k in range(4):
        pm = pass_ms[k] / max(pass_cnt[k], 1)
        per_pass[names[k] if k < 2 or not fused else names[k] + " %d" % k] = {
            "kernel": kern[k], "avg_ms": pm, "alg_bytes": g.pass_bytes(k),
            "GBps": g.pass_bytes(k) / (pm * 1e-3) / 1e9 if pm > 0 and g.pass_bytes(k) > 0 else None}

    # ---- error of the timed configuration against the FP64 oracle (outside the timed region):
    # one step from the bench's own input, sampled Fourier modes, each from the definition
    from oracle import oracle as O
    modes = sampled_modes(n)
    g.set_field(c0_dev)
    g.step(1)
    c1 = g.get_field().cpu().numpy()
    err_ch = mode_error(O.dft_modes(c1, modes, "c"), O.step_modes(c0, modes, DT, MOB, KAPPA, H), field_l2(c1))
    err_ch["k0_rel_err"] = abs(float(np.sum(c1, dtype=np.float64)) - float(np.sum(c0, dtype=np.float64))) / \
        abs(float(np.sum(c0, dtype=np.float64)))
    err_ch["what"] = ("one step from the timed input; c_hat(k) of the GPU field vs the oracle's step evaluated "
                      "mode by mode (direct FP64 sums, no FFT) at %d wave vectors incl. Nyquist and the fastest-"
                      "growing mode; k = 0: FP64 sum of the FP32 field vs the input's" % len(modes))
    del c1

    # ---- Design B: the same timed steps with the fused y-z-y pass (5 sweeps per step;
    # opt-in, since on GB300 it is slower than the three separate passes)
    design_b = None
    if not args.no_design_b and not fused:
        os.environ["EVX_FUSE"] = "1"
        try:
            gb = evx.Grid(shape, dt=DT, M=MOB, kappa=KAPPA, h=H, stream=stream)
        finally:
            os.environ.pop("EVX_FUSE", None)
        if gb.pass_bytes(2) == 0.0:
            gb.set_field(c0_dev)
            gb.step(3)
            gb.set_profiling(True)
            gb.pass_times(reset=True)
            torch.cuda.synchronize()
            e0.record(stream)
            gb.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_b = e0.elapsed_time(e1)
            pm, pc = gb.pass_times(reset=True)
            gb.set_profiling(False)
            gb.set_field(c0_dev)
            gb.step(1)
            c1 = gb.get_field().cpu().numpy()
            design_b = {
                "what": "x pass + fused y inverse/z step/y forward pass whose x slabs stay in L2 (5 sweeps of "
                        "HBM traffic per step instead of 9)",
                "value": job_throughput(1, args.steps, V, ms_b * 1e-3), "unit": UNIT,
                "ms_per_step": ms_b / args.steps, "sweeps_per_step": sum(gb.pass_bytes(k) for k in range(4))
                / field_bytes, "x_pass_ms": pm[0] / max(pc[0], 1), "fused_pass_ms": pm[1] / max(pc[1], 1),
                "fused_kernel": "fused::fyzy_kernel<%d, %d, %d, %d>" % (r1, tp, rz, tz),
                "error_vs_oracle": mode_error(O.dft_modes(c1, modes, "c"),
                                              O.step_modes(c0, modes, DT, MOB, KAPPA, H), field_l2(c1))}
            del c1
        gb.close()

    # ---- end to end through the host API
    e2e = None
    if not args.no_e2e:
        host_in = torch.from_numpy(c0).pin_memory()
        host_out = torch.empty(shape, dtype=torch.float32).pin_memory()
        # one untimed pass through the same buffers: the first transfers from and to
        # freshly pinned pages carry a one-time mapping cost (measured 60-200 ms here)
        g.set_field_host(host_in)
        g.get_field_host(host_out)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.set_field_host(host_in)
        g.step(args.steps)
        g.get_field_host(host_out)
        t1 = time.perf_counter()
        barrier()
        te = max_over_ranks(t1 - t0)
        e2e = {"value": job_throughput(ws, args.steps, V, te), "unit": UNIT,
               "h2d_bytes_per_step": 4.0 * V / args.steps, "d2h_bytes_per_step": 4.0 * V / args.steps,
               "job": "pinned host c0 -> evx_set_field_host -> %d steps -> evx_get_field_host (the result is "
                      "written by the inverse transform straight into the mapped pinned buffer); the field's "
                      "bytes are spread over the job's steps; one untimed pass through the same buffers first"
                      % args.steps}
        del host_in, host_out
    fp = g.footprint()  # the Cahn-Hilliard workload's footprint (the VM model adds a buffer)
    # ---- the Allen-Cahn model on the same engine and grid (device-resident)
    ac = None
    if args.ac_steps > 0:
        g.set_model("ac")
        g.set_field(c0_dev)
        g.step(3)
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        g.step(args.ac_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        t_ac = max_over_ranks(e0.elapsed_time(e1))
        ac = {"workload": "Allen-Cahn %d^3, same c0, dt 0.1, L = kappa = 1, %d steps (after 3 warm-up)"
                          % (n, args.ac_steps),
              "value": job_throughput(ws, args.ac_steps, V, t_ac * 1e-3), "unit": UNIT,
              "ms_per_step": t_ac / args.ac_steps, "launches_per_step": 3 if fused else 5,
              "mean_after": g.mean()}
        g.set_field(c0_dev)
        g.step(1)
        c1 = g.get_field().cpu().numpy()
        ac["error_vs_oracle"] = mode_error(O.dft_modes(c1, modes, "c"),
                                           O.ac_step_modes(c0, modes, DT, MOB, KAPPA, H), field_l2(c1))
        ac["error_vs_oracle"]["mean_abs_err"] = abs(g.mean() - float(np.real(O.ac_step_modes(
            c0, np.zeros((1, 3), dtype=np.int64), DT, MOB, KAPPA, H)[0])) / V)
        ac["error_vs_oracle"]["what"] = "one step, sampled modes as for the CH line; FP64 mean vs the oracle's"
        del c1
        g.set_model("ch")
    # ---- variable-mobility Cahn-Hilliard (FD right-hand side, spectral preconditioner)
    vm = None
    if args.vm_steps > 0:
        g.set_model("vm")
        g.set_field(c0_dev)
        g.step(2)
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        g.step(args.vm_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        t_vm = max_over_ranks(e0.elapsed_time(e1))
        vm = {"workload": "variable-mobility CH %d^3, M(c) = max(1 - c^2, 0), same c0, dt 0.1, kappa = 1, "
                          "%d steps (after 2 warm-up)" % (n, args.vm_steps),
              "value": job_throughput(ws, args.vm_steps, V, t_vm * 1e-3), "unit": UNIT,
              "ms_per_step": t_vm / args.vm_steps,
              # the two stencils run as one kernel when ny % 8 == 0 and nz % 64 == 0
              "launches_per_step": 6 if n % 64 == 0 else 7,
              "footprint_bytes": g.footprint()}
        g.set_field(c0_dev)
        g.step(1)
        c1 = g.get_field().cpu().numpy()
        vm["error_vs_oracle"] = mode_error(O.dft_modes(c1, modes, "c"),
                                           O.vm_step_modes(c0, modes, DT, MOB, KAPPA, H), field_l2(c1))
        vm["error_vs_oracle"]["what"] = ("one step, sampled modes; the oracle's FD right-hand side is formed "
                                         "plane by plane and summed mode by mode")
        del c1
        g.set_model("ch")
    g.close()
    del c0_dev
    torch.cuda.empty_cache()
    sur = None
    if not args.no_surrogate and args.n == 1024:
        try:
            sur = surrogate_bench(args)
        except Exception as ex:  # report, do not fail the bench
            sur = {"error": repr(ex)}

    adj = None
    if not args.no_small and args.n == 1024:
        try:
            adj = adjoint_bench()
        except Exception as ex:  # report, do not fail the bench
            adj = {"error": repr(ex)}
    small = None
    if not args.no_small and args.n == 1024:
        try:
            small = small_grid_bench()
        except Exception as ex:  # report, do not fail the bench
            small = {"error": repr(ex)}
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline_oracle()
        except Exception as ex:  # report, do not fail the bench
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle",
                   "sample": "failed: %r" % (ex,)}
        try:
            cpu["single_thread"] = cpu_single_thread_oracle()
        except Exception as ex:  # report, do not fail the bench
            cpu["single_thread"] = {"value": None, "sample": "failed: %r" % (ex,)}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "CH 3D periodic %d^3, c0 = 0.3 + U(-0.05,0.05) seed 0, dt 0.1, "
                               "M = kappa = 1, h = 1, %d steps" % (n, args.steps),
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "l2": "inputs larger than L2 (%.2f GB per field vs 129 MB)" % (field_bytes / 1e9),
                   "sweeps_per_step": step_bytes / field_bytes,
                   "sweeps_note": ("x pass 3 (read W, S; write S) + fused y-z-y pass 2 (read S, write W; "
                                   "the slab's intermediate sweeps stay in L2)" if fused else
                                   "x pass 3 + y inverse 2 + z step 2 + y forward 2"),
                   "footprint_bytes": fp},
        "error_vs_oracle": err_ch,
        "design_b": design_b,
        "roofline": {"bound": "hbm", "kernel": kern[dom] + " (" + names[dom] + ")",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": peak_src + " hbm_gbs (copy)",
                     "traffic": measured_traffic(dom, alg_bytes),
                     "traffic_source": "profiles/traffic_1024x1024x256.md (ratio scaled to this launch)",
                     "alg_bytes_per_launch": alg_bytes, "avg_ms": avg_ms,
                     "step_alg_bytes": step_bytes,
                     "step_effective_GBps": step_bytes / (t_max / args.steps * 1e-3) / 1e9,
                     "per_pass": per_pass},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": (2 if fused else 4) * args.steps,
        "allen_cahn": ac,
        "variable_mobility": vm,
        "small_grids": small,
        "adjoint": adj,
        "surrogate": sur,
    }
    print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
