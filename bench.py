"""TSQR benchmark on GB300: one JSON line.

A step is one pass of the whole path over one synthetic matrix: tsqr_factor (leaves, flat
chains, tree, root signs), tsqr_form_q (explicit thin Q) and tsqr_apply_qt on one right-hand
side.  The workload: m = 2^22, n = 64, FP64, A = U Sigma V^T with Haar U, V and kappa = 1
(seeded, synthetic).  The metric is GFLOP/s with LAPACK operation counts
(factor 2mn^2 - 2n^3/3, thin Q 2mn^2 - 2n^3/3, Q^T b 4mn - 2n^2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (plain Householder QR + thin Q) on the host cores,
on a bounded slice of the same workload.  Under torchrun each rank runs an independent replica
(TSQR on one GPU needs no data-path collective); value is the sum over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

M_DEFAULT, N_DEFAULT = 1 << 22, 64
METRIC = "TSQR GFLOP/s (factor + thin Q + Q^T b, FP64) at stated ||A-QR||, ||I-Q^TQ|| vs plain FP64"


def flops(m, n, k=1):
    f = 2.0 * m * n * n - 2.0 * n ** 3 / 3
    return {"factor": f, "form_q": f, "apply_qt": 4.0 * m * n * k - 2.0 * n * n * k}


def algorithmic_bytes(m, n, k=1):
    # factor: read A, write V; thin Q: read V, write Q; Q^T b: read V, read+write b
    return {"factor": 16.0 * m * n, "form_q": 16.0 * m * n, "apply_qt": 8.0 * m * n + 16.0 * m * k}


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (the slowest replica's time); x itself without a process
    group.  Every rank gets the result."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def launches_per_step(panels, depth, precision, f32, np_, leaf_h, leaves, chains):
    """Kernels of one step (factor, thin Q, Q^T b with one column): the factorization, one thin-Q
    launch per tree level plus the chain launch, and one Q^T b launch; with P > 1 panels (n > 64)
    also the staging copy, the trailing updates and the earlier panels' Q applied to the later
    column blocks.  For one panel: FP32 storage first widens A into the staging slots, and the
    tensor-core thin Q (modes 2 and 3, FP32 storage; padded width 64, leaves of at most 128 rows)
    runs its chains as three launches: recurrences, first leaves and leaf products (the last is
    skipped when every leaf starts a chain).  With P > 1 the count is the FP64 schedule's."""
    P, d = panels, depth
    n_launch = (P > 1) + P + (P - 1) + P * (d + 1) + (P - 1) * (d + 1) + P
    if P == 1:
        n_launch += int(f32)
        if (precision in (2, 3) or f32) and np_ == 64 and leaf_h <= 128:
            n_launch += 2 if leaves > chains else 1
    return n_launch


def job_value(units_per_step_per_rank, world, ms_per_step):
    """Whole-job throughput: every rank processes the same units per step (weak scaling), and the
    job's step time is the slowest rank's."""
    return units_per_step_per_rank * world / (ms_per_step / 1e3) / 1e9


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# DRAM bytes (read + write) of one factor_kernel<ArithF64> launch, from an ncu capture at
# m = 524288, n = 64 (699.4 MB: 269.0 MB read, 430.3 MB written; taken after the chain step's
# packed dot products), scaled by rows to m = 4194304: A is read once and V and T are written
# once, so traffic grows in proportion to m.  Only valid for the kernel as captured.
FACTOR_F64_TRAFFIC = {(4194304, 64): 8 * 699.37e6}

# FP64 pipe of GB300: 152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz (nominal 1.25 TFLOP/s);
# the fallback when the live probe below cannot run.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

# Thin-Q tensor-core products per useful FP64 multiply-add: the Ozaki split runs 34 bf16 digit
# products (7 balanced base-256 digits, pairs of weight <= 9), bf16x3 six term products (on the
# chains' Y M; the FP32 form's T C stays on the FP32 pipe).
OZAKI_PRODUCTS, BF16X3_PRODUCTS = 34, 6


def measure_pipe_peaks():
    """FP64 and FP32 FMA rates of this GPU in TFLOP/s, measured now by the probe library
    (independent FMA chains on every SM); None where the probe cannot run."""
    import ctypes

    from paper_0809_2407_gb300 import build

    try:
        lib = ctypes.CDLL(build.PROBE_LIB)
    except OSError:
        return {"fp64_tflops": None, "fp32_tflops": None}
    lib.tsqr_probe_fma_tflops.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double)]
    out = {}
    for name, fp32, iters in (("fp64_tflops", 0, 20000), ("fp32_tflops", 1, 1000000)):
        v = ctypes.c_double(0.0)
        out[name] = v.value if lib.tsqr_probe_fma_tflops(fp32, iters, ctypes.byref(v)) == 0 else None
    out["how"] = ("8 independent FMA chains per thread, 8 blocks x 256 threads per SM, CUDA events over the "
                  "second of two launches (about 0.1 s each)")
    # FP64 with 1, 2, 4, 8 warps per SM: what a single warp can issue (the blocked factor's panel
    # runs on one warp)
    lib.tsqr_probe_fma_tflops_warps.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                                                ctypes.POINTER(ctypes.c_double)]
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    byw = {"how": "one block of 32 x warps threads per SM, 8 independent FP64 FMA chains per thread; lanes per "
                  "clock at the 2.07 GHz maximum SM clock"}
    for w in (1, 2, 4, 8):
        v = ctypes.c_double(0.0)
        if lib.tsqr_probe_fma_tflops_warps(0, w, 20000 * 8 // w, ctypes.byref(v)) == 0:
            byw["warps_%d" % w] = {"tflops": v.value, "fma_lanes_per_clock_per_sm": v.value * 1e12 / 2 / sms / 2.07e9}
    out["fp64_by_warps_per_sm"] = byw
    return out


def form_roofline(kind, fl, kernel_ms, ab, peaks, pipes):
    """Roofline of one precision form's step: the dominant kernel against the unit that binds it
    (FP64 pipe for native FP64, FP32 pipe for FP32 storage and double-float arithmetic), with its
    HBM view; for forms whose thin Q runs on the tensor cores, that kernel's tensor view: the bf16
    slice or term products it executes (useful flops x products per multiply-add) against the
    measured bf16 peak."""
    dom = max(("factor", "form_q"), key=lambda k: kernel_ms[k])
    t = kernel_ms[dom] / 1e3
    achieved = fl[dom] / t / 1e12
    if kind in ("fp64", "ozaki_wy", "ozaki_wy_blocked"):
        measured = pipes.get("fp64_tflops")
        peak, src = measured or FP64_PEAK_TFLOPS, "FP64 pipe"
    else:
        measured = pipes.get("fp32_tflops")
        peak, src = measured, "FP32 pipe"
        if kind in ("double_float", "df_ozaki_wy"):
            src += ", useful FP64-equivalent flops (a double-float multiply-add takes about 10 FP32 instructions)"
    src += ": measured in this run" if measured else ": nominal"
    hbm = peaks.get("hbm_gbs")
    r = {"bound": "alu", "kernel": dom + "_kernel", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
         "frac": (achieved / peak) if peak else None, "peak_source": src,
         "hbm_view": {"achieved_gbs": ab[dom] / t / 1e9, "peak_gbs": hbm,
                      "frac_of_measured": (ab[dom] / t / 1e9 / hbm) if hbm else None}}
    prod = {"ozaki_wy": OZAKI_PRODUCTS, "df_ozaki_wy": OZAKI_PRODUCTS, "ozaki_wy_blocked": OZAKI_PRODUCTS,
            "fp32": BF16X3_PRODUCTS, "fp32_blocked": BF16X3_PRODUCTS}.get(kind)
    bf16 = peaks.get("bf16_tflops")
    if prod:
        tq = kernel_ms["form_q"] / 1e3
        # fp32: the tensor cores take Y M, half of the thin Q's multiply-adds
        share = 0.5 if kind.startswith("fp32") else 1.0
        tc = fl["form_q"] * share * prod / tq / 1e12
        r["tensor_view"] = {"kernel": "form_q (chains)", "products_per_fma": prod, "share_on_tensor_cores": share,
                            "achieved_bf16_tflops": tc, "peak_bf16_tflops": bf16,
                            "frac_of_measured": (tc / bf16) if bf16 else None}
    return r


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_input(m, n):
    from paper_0809_2407_gb300 import inputs

    return inputs.usv(m, n, 0.0, inputs.seed_for(2, 0))


def cpu_oracle_sample(A_h, rows, openmp=False):
    """Times the oracle on the first `rows` rows, the step of the GPU line (QR, thin Q and Q^T b
    through the stored reflectors); returns (GFLOP/s, seconds, threads).  openmp: the oracle's
    -fopenmp build (bitwise the serial results) on all host cores."""
    import numpy as np

    import oracle

    threads = 1
    if openmp:
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
        threads = int(os.environ["OMP_NUM_THREADS"])
        oracle.set_variant("openmp")
    try:
        oracle._load()
        S = A_h[:rows].copy()
        b = np.random.default_rng(5).standard_normal((rows, 1))
        t0 = time.perf_counter()
        res = oracle.qr(S, want_q=True)
        oracle.apply_qt(res["V"], res["tau"], b)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_variant("serial")
    return sum(flops(rows, S.shape[1]).values()) / dt / 1e9, dt, threads


def main_config(m, n, precision, world):
    """The benchmark line's config (shared by the GPU and reference arms)."""
    return {"workload": "tsqr factor + form_q + apply_qt(k=1), fp64, m=%d n=%d, A=U S V^T kappa=1" % (m, n),
            "m": m, "n": n, "k": 1, "leaf_h": None, "chain": "auto", "arity": 2, "precision": precision,
            "l2": "inputs larger than L2 (A is %.1f GB)" % (8.0 * m * n / 1e9),
            "parallelism": "replicas" if world > 1 else "single-gpu"}


def host_cpu():
    """The host's CPU model and core count (context for the CPU lines)."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:  # Arm hosts name the core in lscpu, not in /proc/cpuinfo
        import subprocess

        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    if model is None:
        import platform

        model = platform.machine()
    return {"model": model, "cpu_count": os.cpu_count()}


def cpu_library_sample(torch, A_h, rows):
    """torch.linalg.qr (LAPACK geqrf + orgqr) on the host cores, on the same rows as the oracle's
    sample: a labelled library reference beside the oracle, not a target."""
    X = torch.from_numpy(A_h[:rows].copy())
    torch.linalg.qr(X)
    t0 = time.perf_counter()
    for _ in range(3):
        torch.linalg.qr(X)
    dt = (time.perf_counter() - t0) / 3
    f = flops(rows, A_h.shape[1])
    return {"what": "torch.linalg.qr on the host (LAPACK), explicit Q and R", "threads": torch.get_num_threads(),
            "value": (f["factor"] + f["form_q"]) / dt / 1e9, "unit": "GFLOP/s", "seconds": dt}


def run_reference(args, rank, world):
    """The oracle on host cores, on bounded slices of the workload (rank 0 only)."""
    if rank != 0:
        return None
    m, n = args.m, args.n
    rows = args.ref_rows
    from paper_0809_2407_gb300 import inputs

    A_h = inputs.usv(rows, n, 0.0, inputs.seed_for(2, 0))
    for _ in range(min(args.warmup, 1)):
        cpu_oracle_sample(A_h, rows)
    times = []
    for _ in range(args.steps):
        _, dt, _ = cpu_oracle_sample(A_h, rows)
        times.append(dt)
    per = sum(flops(rows, n).values())
    tot = sum(times)
    value = per * len(times) / tot / 1e9
    return {"metric": METRIC, "value": value, "unit": "GFLOP/s", "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": main_config(m, n, 0, world),
            "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": "oracle QR, thin Q and Q^T b of an A = U S V^T (kappa = 1) of %d rows x %d "
                                       "columns from the workload's generator, per step" % (rows, n)},
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_batched(tsqr, torch, dev, stream, sptr, args, count=512, seed=20084000):
    """512 matrices: m log-uniform in [1e4, 2^18], n from {8, 16, 32, 64}, N(0,1) entries from
    per-matrix seeds (generated on the device).  Times factor + thin Q of all of them: one batched
    launch sequence replayed from a CUDA graph, and a loop of single-matrix calls."""
    import numpy as np

    rng = np.random.default_rng(seed)
    ms = np.floor(np.exp(rng.uniform(np.log(1e4), np.log(2.0 ** 18), count))).astype(np.int64)
    ns = rng.choice([8, 16, 32, 64], count)
    mats = []
    for i in range(count):
        g = torch.Generator(device=dev).manual_seed(seed + i)
        mats.append(torch.randn((int(ms[i]), int(ns[i])), dtype=torch.float64, device=dev, generator=g))
    fl = float(sum(4.0 * m_ * n_ * n_ - 4.0 * n_ ** 3 / 3 for m_, n_ in zip(ms, ns)))
    steps = max(1, min(args.steps, 5))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    big = int(np.argmax(ms))

    def graph_run(batch_mats, plans=None, precision=0):
        """Times the batch's factor + thin Q replayed from a CUDA graph; accuracy of the largest."""
        b = tsqr.Batch(batch_mats, plans=plans, precision=precision)
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            for _ in range(2):
                b.factor()
                b.form_q()
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            b.factor()
            b.form_q()
        for _ in range(2):
            graph.replay()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / steps
        good = b.status() == tsqr.TSQR_OK
        A, Q, R = batch_mats[big].double(), b.Q[big].double(), b.R[big].double()
        acc = ((torch.linalg.norm(A - Q @ R) / torch.linalg.norm(A)).item(),
               torch.linalg.norm(torch.eye(int(ns[big]), dtype=torch.float64, device=dev) - Q.T @ Q).item())
        b.close()
        del b, graph
        torch.cuda.empty_cache()
        return t, good, acc

    ms_batched, ok, (be, orth) = graph_run(mats)
    # plans per padded width tuned on this batch (leaf height and arity; chains shared)
    t_tune = time.perf_counter()
    plans, picked = tsqr.autotune_batch(mats, leaf_hs=(64, 128, 256, 512), arities=(2, 4), reps=1)
    t_tune = time.perf_counter() - t_tune
    ms_tuned, ok_t, (be_t, orth_t) = graph_run(mats, plans)
    # precision forms of the batch: the Ozaki forms' thin Q takes the tensor cores for n = 64
    forms = {}
    for nm, prec in (("double_float", 1), ("ozaki_wy", 2), ("df_ozaki_wy", 3)):
        t_f, ok_f, (be_f, orth_f) = graph_run(mats, None, prec)
        forms[nm] = {"precision": prec, "value": fl / (t_f / 1e3) / 1e9, "unit": "GFLOP/s", "ms_per_step": t_f,
                     "speedup_vs_fp64_batched": ms_batched / t_f, "status_ok": ok_f,
                     "largest": {"backward_error": be_f, "orthogonality": orth_f}}
    mats32 = [A.float() for A in mats]
    ms32, ok32, (be32, orth32) = graph_run(mats32)
    del mats32
    # the same work as a loop of single-matrix launches (workspaces and outputs preallocated)
    items = []
    for A in mats:
        m_, n_ = A.shape
        o = tsqr.Opts()
        nb = tsqr.tsqr_workspace_size(tsqr.TSQR_F64, m_, n_, o)
        items.append((A, torch.empty(nb, dtype=torch.uint8, device=dev), nb,
                      torch.empty((n_, n_), dtype=torch.float64, device=dev),
                      torch.empty((m_, n_), dtype=torch.float64, device=dev), o))

    def loop():
        for A, w, nb, R_, Q_, o in items:
            m_, n_ = A.shape
            h = tsqr.tsqr_factor(tsqr.TSQR_F64, tsqr.TSQR_ROW_MAJOR, m_, n_, A.data_ptr(), n_, R_.data_ptr(), n_,
                                 w.data_ptr(), nb, o, sptr)
            tsqr.tsqr_form_q(h, Q_.data_ptr(), n_, sptr)
            tsqr.tsqr_destroy(h)

    loop()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        loop()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_loop = e0.elapsed_time(e1) / steps
    del items
    return {"matrices": count, "elements": int(sum(int(m_) * int(n_) for m_, n_ in zip(ms, ns))),
            "workload": "m log-uniform in [1e4, 2^18], n in {8,16,32,64}, N(0,1), fp64, factor + thin Q",
            "value": fl / (ms_batched / 1e3) / 1e9, "unit": "GFLOP/s", "ms_per_step": ms_batched,
            "launch": "one persistent factor launch (resident blocks take chains longest first from a device "
                      "queue) + one thin-Q launch per tree depth + one chain launch, CUDA graph; default plans",
            "tuned": {"value": fl / (ms_tuned / 1e3) / 1e9, "unit": "GFLOP/s", "ms_per_step": ms_tuned,
                      "speedup_vs_default_plans": ms_batched / ms_tuned, "status_ok": ok_t,
                      "plans": {"np%d" % w: {"leaf_h": h or "default", "arity": a} for w, (h, a) in picked.items()},
                      "tuning_seconds": t_tune,
                      "how": "autotune_batch: per padded width, coordinate descent over leaf height {64, 128, 256, "
                             "512} and arity {2, 4} timing this batch's factor + thin Q",
                      "largest": {"backward_error": be_t, "orthogonality": orth_t}},
            "forms": forms,
            "loop_value": fl / (ms_loop / 1e3) / 1e9, "loop_ms_per_step": ms_loop,
            "speedup_vs_loop": ms_loop / ms_batched, "status_ok": ok,
            "largest": {"m": int(ms[big]), "n": int(ns[big]), "backward_error": be, "orthogonality": orth},
            "fp32": {"value": fl / (ms32 / 1e3) / 1e9, "unit": "GFLOP/s", "ms_per_step": ms32,
                     "speedup_vs_fp64_batched": ms_batched / ms32, "status_ok": ok32,
                     "note": "the same matrices rounded to float32, FP32 storage and arithmetic, CUDA graph",
                     "largest": {"backward_error": be32, "orthogonality": orth32}}}


def run_e2e(tsqr, torch, dev, stream, sptr, A_pin, b_h, A, Q, R, b, work, nbytes, opts, m, n, steps, world):
    """The step through the C-ABI with host buffers: H2D of A and b from pinned memory, then
    factor, thin Q and Q^T b, then D2H of R, Q and Q^T b, every step.  Timed two ways: serially on
    one stream, and pipelined with two buffer sets, where the copies of neighbouring steps run on
    two copy streams while the current step computes (what a caller streaming matrices does)."""
    per_step = sum(flops(m, n).values())
    R_h = [torch.empty((n, n), dtype=torch.float64).pin_memory() for _ in range(2)]
    Q_h = [torch.empty((m, n), dtype=torch.float64).pin_memory() for _ in range(2)]
    bo_h = [torch.empty((m, 1), dtype=torch.float64).pin_memory() for _ in range(2)]
    Ad, Qd, Rd, bd = [A, torch.empty_like(A)], [Q, torch.empty_like(Q)], [R, torch.empty_like(R)], [b, torch.empty_like(b)]

    def step_on(j, s_ptr):
        h = tsqr.tsqr_factor(tsqr.TSQR_F64, tsqr.TSQR_ROW_MAJOR, m, n, Ad[j].data_ptr(), n, Rd[j].data_ptr(), n,
                             work.data_ptr(), nbytes, opts, s_ptr)
        tsqr.tsqr_form_q(h, Qd[j].data_ptr(), n, s_ptr)
        tsqr.tsqr_apply_qt(h, 1, bd[j].data_ptr(), 1, s_ptr)
        return h

    def serial(K):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            Ad[0].copy_(A_pin, non_blocking=True)
            bd[0].copy_(b_h, non_blocking=True)
            h = step_on(0, sptr)
            R_h[0].copy_(Rd[0], non_blocking=True)
            Q_h[0].copy_(Qd[0], non_blocking=True)
            bo_h[0].copy_(bd[0], non_blocking=True)
            tsqr.tsqr_destroy(h)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K

    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def pipelined(K):
        torch.cuda.synchronize()
        ev_in = [torch.cuda.Event() for _ in range(K)]
        ev_c = [torch.cuda.Event() for _ in range(K)]
        ev_out = [torch.cuda.Event() for _ in range(K)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s_in)
        for i in range(K):
            j = i % 2
            if i >= 2:
                s_in.wait_event(ev_out[i - 2])  # buffers j are free once step i-2's results left
            with torch.cuda.stream(s_in):
                Ad[j].copy_(A_pin, non_blocking=True)
                bd[j].copy_(b_h, non_blocking=True)
            ev_in[i].record(s_in)
            stream.wait_event(ev_in[i])
            h = step_on(j, sptr)
            ev_c[i].record(stream)
            s_out.wait_event(ev_c[i])
            with torch.cuda.stream(s_out):
                R_h[j].copy_(Rd[j], non_blocking=True)
                Q_h[j].copy_(Qd[j], non_blocking=True)
                bo_h[j].copy_(bd[j], non_blocking=True)
            ev_out[i].record(s_out)
            tsqr.tsqr_destroy(h)
        e1.record(s_out)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K

    serial(1)
    ser_ms = serial(max(1, min(steps, 3)))
    pipelined(2)
    K = max(3, min(steps, 10))
    pipe_ms = pipelined(K)
    ok = bool(torch.equal(Q_h[0], Q_h[1]) and torch.equal(R_h[0], R_h[1]))
    return {"value": per_step * world / (pipe_ms / 1e3) / 1e9, "unit": "GFLOP/s",
            "h2d_bytes_per_step": 8 * m * n + 8 * m, "d2h_bytes_per_step": 8 * n * n + 8 * m * n + 8 * m,
            "ms_per_step": pipe_ms, "steps": K,
            "schedule": "pipelined: two device buffer sets; step i+1's H2D and step i-1's D2H run on two copy "
                        "streams while step i computes; timed from the first H2D to the last D2H",
            "results_identical_across_buffers": ok,
            "serial": {"value": per_step * world / (ser_ms / 1e3) / 1e9, "ms_per_step": ser_ms,
                       "schedule": "one stream: H2D, factor, thin Q, Q^T b, D2H"}}


SHAPE_FORMS = {32: (("double_float", 1, False), ("fp32", 0, True)),
               128: (("double_float", 1, False), ("ozaki_wy", 2, False), ("df_ozaki_wy", 3, False),
                     ("fp32", 0, True))}


def time_form(tsqr, torch, dev, stream, sptr, A, m, n, precision, f32, steps=3, warmup=2, leaf_h=0):
    """One step (factor, thin Q, Q^T b) of one precision form on the device matrix A, timed per
    kernel with CUDA events; GFLOP/s with the LAPACK counts, backward error and orthogonality."""
    import numpy as np

    code = tsqr.TSQR_F32 if f32 else tsqr.TSQR_F64
    A_ = A.float() if f32 else A
    b = torch.from_numpy(np.random.default_rng(6).standard_normal((m, 1))).to(dev).to(A_.dtype)
    Q = torch.empty((m, n), dtype=A_.dtype, device=dev)
    R = torch.empty((n, n), dtype=A_.dtype, device=dev)
    opts = tsqr.Opts(precision=precision, leaf_h=leaf_h)
    nbytes = tsqr.tsqr_workspace_size(code, m, n, opts)
    work = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    ev = {"factor": [], "form_q": [], "apply_qt": []}
    for it in range(warmup + steps):
        mk = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        mk[0].record(stream)
        h = tsqr.tsqr_factor(code, tsqr.TSQR_ROW_MAJOR, m, n, A_.data_ptr(), n, R.data_ptr(), n,
                             work.data_ptr(), nbytes, opts, sptr)
        mk[1].record(stream)
        tsqr.tsqr_form_q(h, Q.data_ptr(), n, sptr)
        mk[2].record(stream)
        tsqr.tsqr_apply_qt(h, 1, b.data_ptr(), 1, sptr)
        mk[3].record(stream)
        info = tsqr.tsqr_handle_info(h)
        tsqr.tsqr_destroy(h)
        torch.cuda.synchronize()
        if it >= warmup:
            for i, k in enumerate(("factor", "form_q", "apply_qt")):
                ev[k].append(mk[i].elapsed_time(mk[i + 1]))
    fl = flops(m, n)
    ms = sum(statistics.mean(v) for v in ev.values())
    Ad, Qd, Rd = A_.double(), Q.double(), R.double()
    res = {"m": m, "n": n, "panels": info.panels, "leaf_h": info.leaf_h, "chains": info.chains,
           "value": sum(fl.values()) / (ms / 1e3) / 1e9, "unit": "GFLOP/s", "ms_per_step": ms,
           "kernel_ms": {k: statistics.mean(v) for k, v in ev.items()},
           "backward_error": (torch.linalg.norm(Ad - Qd @ Rd) / torch.linalg.norm(Ad)).item(),
           "orthogonality": torch.linalg.norm(torch.eye(n, dtype=torch.float64, device=dev) - Qd.T @ Qd).item()}
    del Ad, Qd, Rd, A_, b, Q, R, work
    torch.cuda.empty_cache()
    return res



def run_shapes(tsqr, torch, dev, stream, sptr, m, ns=(16, 32, 128), steps=3, warmup=2, forms=SHAPE_FORMS):
    """Plain FP64 TSQR (factor + thin Q + Q^T b) on the other column counts of the workload
    family, A = U Sigma V^T with kappa = 1: n = 16 and 32 are single TSQRs with taller leaves,
    n = 128 is the blocked QR over two 64-column TSQR panels.  The precision forms run beside
    FP64 at n = 32 and 128 (the Ozaki forms only differ from FP64 where np = 64: at n = 128 the
    panels' thin Q and their trailing updates Q^T [A_2] and Q [0; Q_2] run on the tensor cores)."""
    out = {}
    for n in ns:
        A = torch.from_numpy(make_input(m, n)).to(dev)
        out["n%d" % n] = time_form(tsqr, torch, dev, stream, sptr, A, m, n, 0, False, steps, warmup)
        if forms and n in forms:
            f64_ms = out["n%d" % n]["ms_per_step"]
            out["n%d" % n]["forms"] = {}
            for name, precision, f32 in forms[n]:
                r = time_form(tsqr, torch, dev, stream, sptr, A, m, n, precision, f32, steps, warmup)
                r["speedup_vs_f64"] = f64_ms / r["ms_per_step"]
                out["n%d" % n]["forms"][name] = r
        del A
        torch.cuda.empty_cache()
    return out


def run_tree_levels(tsqr, torch, dev, stream, sptr, n=64, levels=(3, 4, 5, 6, 7), reps=5):
    """Time per level of the reduction tree: 2^L chains of one 64-row leaf each under a binary
    tree of L levels (at most 128 chains, so the leaves run as one wave on the GPU's SMs; the
    levels run one after another, each a structured node step per pair), factor time against L;
    the slope is the time per level."""
    import numpy as np

    pts = []
    for L in levels:
        m = 64 * (1 << L)
        A = torch.from_numpy(np.random.default_rng(9).standard_normal((m, n))).to(dev)
        R = torch.empty((n, n), dtype=torch.float64, device=dev)
        o = tsqr.Opts(leaf_h=64, chain=1, arity=2)
        nb = tsqr.tsqr_workspace_size(tsqr.TSQR_F64, m, n, o)
        w = torch.empty(nb, dtype=torch.uint8, device=dev)
        ts = []
        for it in range(reps + 2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h = tsqr.tsqr_factor(tsqr.TSQR_F64, tsqr.TSQR_ROW_MAJOR, m, n, A.data_ptr(), n, R.data_ptr(), n,
                                 w.data_ptr(), nb, o, sptr)
            e1.record(stream)
            tsqr.tsqr_destroy(h)
            torch.cuda.synchronize()
            if it >= 2:
                ts.append(e0.elapsed_time(e1))
        pts.append((L, min(ts)))
        del A, R, w
    x = np.array([p[0] for p in pts], dtype=float)
    y = np.array([p[1] for p in pts])
    slope = float(np.polyfit(x, y, 1)[0])
    return {"ms_per_level": slope, "n": n, "points_ms": {"levels_%d" % L: t for L, t in pts},
            "how": "factor of 2^L x 64 rows as 2^L one-leaf chains under a binary tree of L levels (FP64); "
                   "least-squares slope of time against L"}


COND_FORMS = (("fp64", 0, False), ("double_float", 1, False), ("ozaki_wy", 2, False), ("df_ozaki_wy", 3, False),
              ("fp32", 0, True))


def run_conditioning(tsqr, torch, dev, stream, sptr, m, n, steps=2, warmup=1):
    """Every precision form on the conditioning inputs of the workload family at the benchmark's
    size: A = U Sigma V^T with kappa = 1e4, 1e6, 1e8 and 1e12 (U, V as the main line's) and the
    s-step monomial Krylov basis of a random sparse symmetric matrix.  The Krylov basis is
    numerically rank deficient, and at kappa = 1e12 R is not unique to the working precision, so
    there only the backward error and orthogonality, which Householder QR bounds whatever the
    conditioning, are meaningful."""
    from paper_0809_2407_gb300 import inputs

    ks = (4.0, 6.0, 8.0, 12.0)

    def mats():
        for k, Ah in zip(ks, inputs.usv_family(m, n, ks, inputs.seed_for(2, 0))):
            yield "usv_kappa_1e%d" % int(k), Ah
        yield "krylov", inputs.krylov(m, n, inputs.seed_for(2, 50))

    out = {"m": m, "n": n, "steps": steps, "inputs": "A = U Sigma V^T, singular values log-spaced from 1 to 1/kappa; "
           "krylov: [x, Sx, ...] with unit columns, S sparse symmetric (about 8 nonzeros per row) scaled "
           "to spectral radius 1"}
    for name, Ah in mats():
        A = torch.from_numpy(Ah).to(dev)
        del Ah
        row = {}
        for fname, precision, f32 in COND_FORMS:
            r = time_form(tsqr, torch, dev, stream, sptr, A, m, n, precision, f32, steps, warmup)
            row[fname] = {k: r[k] for k in ("value", "unit", "ms_per_step", "kernel_ms", "backward_error",
                                            "orthogonality")}
        out[name] = row
        del A
        torch.cuda.empty_cache()
    return out


def run_apply_wide(tsqr, torch, dev, stream, sptr, A, m, n, k=64, steps=3):
    """Q^T B then Q B for a 64-column B on one factorization of A, per form: 4mnk - 2n^2k flops
    each way (the LAPACK count of applying n reflectors to k columns)."""
    import numpy as np

    out = {"k": k, "flops_each_way": 4.0 * m * n * k - 2.0 * n * n * k}
    B_h = torch.from_numpy(np.random.default_rng(7).standard_normal((m, k)))
    for name, precision, f32 in (("fp64", 0, False), ("ozaki_wy", 2, False), ("df_ozaki_wy", 3, False),
                                 ("fp32", 0, True)):
        code = tsqr.TSQR_F32 if f32 else tsqr.TSQR_F64
        dt = torch.float32 if f32 else torch.float64
        A_ = A.to(dt)
        R = torch.empty((n, n), dtype=dt, device=dev)
        B0 = B_h.to(dt).to(dev)
        B = B0.clone()
        opts = tsqr.Opts(precision=precision)
        nbytes = tsqr.tsqr_workspace_size(code, m, n, opts)
        work = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        h = tsqr.tsqr_factor(code, tsqr.TSQR_ROW_MAJOR, m, n, A_.data_ptr(), n, R.data_ptr(), n,
                             work.data_ptr(), nbytes, opts, sptr)
        tq, tqt = [], []
        for it in range(1 + steps):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            tsqr.tsqr_apply_qt(h, k, B.data_ptr(), k, sptr)
            e[1].record(stream)
            tsqr.tsqr_apply_q(h, k, B.data_ptr(), k, sptr)
            e[2].record(stream)
            torch.cuda.synchronize()
            if it:
                tqt.append(e[0].elapsed_time(e[1]))
                tq.append(e[1].elapsed_time(e[2]))
        err = ((B - B0).abs().max() / B0.abs().max()).item()  # Q Q^T B = B
        tsqr.tsqr_destroy(h)
        a, b = statistics.mean(tqt), statistics.mean(tq)
        out[name] = {"apply_qt_ms": a, "apply_q_ms": b,
                     "value": 2 * out["flops_each_way"] / ((a + b) / 1e3) / 1e9, "unit": "GFLOP/s",
                     "roundtrip_rel_err": err}
        del A_, R, B0, B, work
        torch.cuda.empty_cache()
    return out


def run_autograd(tsqr, torch, dev, args, batch=64, m=65536, n=32, seed=20085000):
    """Forward + backward of sum(W1*Q) + sum(W2*R) for a batch of 64 matrices of 65536 x 32
    (FP64, and the same data rounded to FP32): time and peak extra memory when the backward keeps
    the implicit Q tree, when it recomputes it from A, and for torch.linalg.qr (cuSOLVER and its
    autograd, which keeps an explicit Q) as a library reference."""
    g = torch.Generator(device=dev).manual_seed(seed)
    A0 = torch.randn((batch, m, n), dtype=torch.float64, device=dev, generator=g)
    W1 = torch.randn((batch, m, n), dtype=torch.float64, device=dev, generator=g)
    W2 = torch.randn((batch, n, n), dtype=torch.float64, device=dev, generator=g)
    out = {"workload": "batch of %d x %d x %d, fp64 and fp32, loss sum(W1*Q)+sum(W2*R)" % (batch, m, n)}
    grads = {}
    A032, W132, W232 = A0.float(), W1.float(), W2.float()

    def step(kind):
        f32 = kind.endswith("_fp32")
        A = (A032 if f32 else A0).detach().clone().requires_grad_(True)
        if kind.startswith("torch"):
            Q, R = torch.linalg.qr(A)
        else:
            Q, R = tsqr.qr_autograd(A, keep=kind.replace("_fp32", ""))
        L = ((W132 if f32 else W1) * Q).sum() + ((W232 if f32 else W2) * R).sum()
        L.backward()
        return A.grad

    for kind in ("tree", "recompute", "torch", "tree_fp32", "torch_fp32"):
        step(kind)
        torch.cuda.synchronize()
        base = torch.cuda.memory_allocated(dev)
        torch.cuda.reset_peak_memory_stats(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 2
        e0.record()
        for _ in range(reps):
            grads[kind] = step(kind)
        e1.record()
        torch.cuda.synchronize()
        out[kind] = {"ms_per_step": e0.elapsed_time(e1) / reps,
                     "peak_extra_bytes": torch.cuda.max_memory_allocated(dev) - base}
    # the two TSQR backward variants agree bitwise; against cuSOLVER's QR (same sign convention
    # after normalising diag(R) >= 0 is not guaranteed there), compare gradient norms only
    out["tree_equals_recompute"] = bool(torch.equal(grads["tree"], grads["recompute"]))
    out["grad_norm_tsqr"] = torch.linalg.norm(grads["tree"]).item()
    out["fp32_grad_rel_diff_vs_fp64"] = (torch.linalg.norm(grads["tree_fp32"].double() - grads["tree"]) /
                                         torch.linalg.norm(grads["tree"])).item()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--m", type=int, default=M_DEFAULT)
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--ref-rows", type=int, default=1 << 15, help="oracle rows per reference-arm step")
    ap.add_argument("--cpu-rows", type=int, default=1 << 17, help="oracle rows of the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip timing the precision forms")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-matrix batched workload")
    ap.add_argument("--no-autograd", action="store_true", help="skip the differentiable-QR workload")
    ap.add_argument("--no-shapes", action="store_true", help="skip the n = 16, 32, 128 shapes")
    ap.add_argument("--no-conditioning", action="store_true",
                    help="skip the kappa = 1e4..1e12 and Krylov inputs (every precision form)")
    ap.add_argument("--apply-wide", action="store_true",
                    help="time Q^T B / Q B with 64 columns even with --no-forms (for profiling)")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2, 3],
                    help="arithmetic mode of the main line (0 native FP64; 1 and 2 are for profiling)")
    ap.add_argument("--fp32", action="store_true", help="main line in FP32 storage (for profiling)")
    ap.add_argument("--leaf-h", type=int, default=0,
                    help="leaf height of the main line (64 selects the blocked tensor-core factor step of "
                         "precision 2 and FP32 storage; for profiling)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return

    import numpy as np
    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    from paper_0809_2407_gb300 import build, tsqr

    build.build()
    tsqr.load()

    m, n = args.m, args.n
    A_h = make_input(m, n)
    A_pin = torch.from_numpy(A_h).pin_memory()
    A = A_pin.to(dev, non_blocking=False)
    b_h = torch.from_numpy(np.random.default_rng(5).standard_normal((m, 1))).pin_memory()
    b = b_h.to(dev)  # Q^T is applied to it in place every step; it stays a unit-scale vector
    Q = torch.empty((m, n), dtype=torch.float64, device=dev)
    R = torch.empty((n, n), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    sptr = tsqr.ctypes.c_void_p(stream.cuda_stream)
    work_holder = {}

    def run_mode(precision, steps, warmup, sample_clocks, f32=False, leaf_h=0):
        """Times `steps` full steps in one arithmetic mode (f32: FP32 storage, the float32
        rounding of the same A; leaf_h: 64 selects the blocked tensor-core factor step of mode 2
        and FP32 storage); returns timings and accuracy."""
        opts = tsqr.Opts(precision=precision, leaf_h=leaf_h)
        code = tsqr.TSQR_F32 if f32 else tsqr.TSQR_F64
        if f32:
            A_, Q_, R_, b_ = A.float(), Q.float(), R.float(), b.float()
        else:
            A_, Q_, R_, b_ = A, Q, R, b
        nbytes = tsqr.tsqr_workspace_size(code, m, n, opts)
        if work_holder.get("bytes", 0) < nbytes:
            work_holder.pop("t", None)
            torch.cuda.empty_cache()
            work_holder["t"] = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            work_holder["bytes"] = nbytes
        work = work_holder["t"]

        def step(record):
            marks = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if record else None
            if record:
                marks[0].record(stream)
            h = tsqr.tsqr_factor(code, tsqr.TSQR_ROW_MAJOR, m, n, A_.data_ptr(), n, R_.data_ptr(), n,
                                 work.data_ptr(), nbytes, opts, sptr)
            if record:
                marks[1].record(stream)
            tsqr.tsqr_form_q(h, Q_.data_ptr(), n, sptr)
            if record:
                marks[2].record(stream)
            tsqr.tsqr_apply_qt(h, 1, b_.data_ptr(), 1, sptr)
            if record:
                marks[3].record(stream)
            tsqr.tsqr_destroy(h)
            return marks

        for _ in range(warmup):
            step(False)
        h = tsqr.tsqr_factor(code, tsqr.TSQR_ROW_MAJOR, m, n, A_.data_ptr(), n, R_.data_ptr(), n,
                             work.data_ptr(), nbytes, opts, sptr)
        info = tsqr.tsqr_handle_info(h)
        tsqr.tsqr_destroy(h)
        launches = launches_per_step(info.panels, info.depth, precision, f32, info.np, info.leaf_h, info.leaves,
                                     info.chains)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        sampler = ClockSampler(local) if (rank == 0 and sample_clocks) else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        all_marks = [step(True) for _ in range(steps)]
        t1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        ms = t0.elapsed_time(t1)
        ev = {"factor": [mk[0].elapsed_time(mk[1]) for mk in all_marks],
              "form_q": [mk[1].elapsed_time(mk[2]) for mk in all_marks],
              "apply_qt": [mk[2].elapsed_time(mk[3]) for mk in all_marks]}
        ms = max_over_ranks(ms, dist, dev)
        Ad, Qd, Rd = A_.double(), Q_.double(), R_.double()
        be = (torch.linalg.norm(Ad - Qd @ Rd) / torch.linalg.norm(Ad)).item()
        orth = torch.linalg.norm(torch.eye(n, dtype=torch.float64, device=dev) - Qd.T @ Qd).item()
        del Ad, Qd, Rd
        return {"ms": ms, "ev": ev, "be": be, "orth": orth, "clocks": clocks, "opts": opts, "nbytes": nbytes,
                "launches": launches}

    pipes = measure_pipe_peaks()
    main_mode = run_mode(args.precision, args.steps, args.warmup, True, f32=args.fp32, leaf_h=args.leaf_h)
    # end to end right after the main line, before the other sections fill host and device memory
    e2e = None
    if not args.no_e2e and not args.fp32:
        e2e = run_e2e(tsqr, torch, dev, stream, sptr, A_pin, b_h, A, Q, R, b, work_holder["t"],
                      main_mode["nbytes"], main_mode["opts"], m, n, args.steps, world)
    ms = main_mode["ms"]
    ev = main_mode["ev"]
    clocks = main_mode["clocks"]
    be, orth = main_mode["be"], main_mode["orth"]
    opts = main_mode["opts"]
    nbytes = main_mode["nbytes"]
    work = work_holder["t"]

    fl = flops(m, n)
    per_step = sum(fl.values())
    ms_step = ms / args.steps
    value = job_value(per_step, world, ms_step)

    # roofline of the dominant kernel (the factorization): FP64-pipe bound
    f_ms = statistics.mean(ev["factor"])
    q_ms = statistics.mean(ev["form_q"])
    a_ms = statistics.mean(ev["apply_qt"])
    dom = "factor" if f_ms >= q_ms else "form_q"
    dom_ms = f_ms if dom == "factor" else q_ms
    achieved_tf = fl[dom] / (dom_ms / 1e3) / 1e12
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs")
    ab = algorithmic_bytes(m, n)
    fp64_peak = pipes.get("fp64_tflops") or FP64_PEAK_TFLOPS
    roofline = {"bound": "alu", "kernel": dom + "_kernel", "achieved": achieved_tf, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": achieved_tf / fp64_peak,
                "traffic": FACTOR_F64_TRAFFIC.get((m, n))
                if (dom == "factor" and args.precision == 0 and not args.fp32 and args.leaf_h == 0) else None,
                "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                "peak_source": ("FP64 pipe, measured in this run by the FMA-chain probe (%s); nominal 152 SMs x 2 "
                                "DFMA/clk x 2.07 GHz = %.3f TFLOP/s" % (pipes.get("how"), FP64_PEAK_TFLOPS))
                if pipes.get("fp64_tflops") else "FP64 pipe, 152 SMs x 2 DFMA/clk x 2.07 GHz (nominal 1.25 TFLOP/s)",
                "measured_pipes": pipes,
                "hbm_view": {"achieved_gbs": ab[dom] / (dom_ms / 1e3) / 1e9, "peak_gbs": hbm,
                             "frac_of_measured": (ab[dom] / (dom_ms / 1e3) / 1e9 / hbm) if hbm else None}}

    # precision forms on the same workload (reported beside the plain FP64 line)
    forms = {}
    if not args.no_forms:
        dfm = run_mode(1, args.steps, min(args.warmup, 3), False)
        d_ms = dfm["ms"] / args.steps
        forms["double_float"] = {
            "precision": 1, "dtype": "f32x2", "value": per_step * world / (d_ms / 1e3) / 1e9, "unit": "GFLOP/s",
            "ms_per_step": d_ms, "speedup_vs_f64": ms_step / d_ms,
            "kernel_ms": {k: statistics.mean(v) for k, v in dfm["ev"].items()},
            "backward_error": dfm["be"], "orthogonality": dfm["orth"]}
        ozm = run_mode(2, args.steps, min(args.warmup, 3), False)
        o_ms = ozm["ms"] / args.steps
        forms["ozaki_wy"] = {
            "precision": 2, "dtype": "f64+bf16x7-digit-split", "value": per_step * world / (o_ms / 1e3) / 1e9,
            "unit": "GFLOP/s", "ms_per_step": o_ms, "speedup_vs_f64": ms_step / o_ms,
            "kernel_ms": {k: statistics.mean(v) for k, v in ozm["ev"].items()},
            "backward_error": ozm["be"], "orthogonality": ozm["orth"],
            "note": "native FP64 reflectors, T merges and tree; the factor's Gram entries and the thin-Q products "
                    "T*C and Y*M on tcgen05 tensor cores as Ozaki splits (7 balanced base-256 digits)"}
        dzm = run_mode(3, args.steps, min(args.warmup, 3), False)
        dz_ms = dzm["ms"] / args.steps
        forms["df_ozaki_wy"] = {
            "precision": 3, "dtype": "f32x2+bf16x7-digit-split", "value": per_step * world / (dz_ms / 1e3) / 1e9,
            "unit": "GFLOP/s", "ms_per_step": dz_ms, "speedup_vs_f64": ms_step / dz_ms,
            "kernel_ms": {k: statistics.mean(v) for k, v in dzm["ev"].items()},
            "backward_error": dzm["be"], "orthogonality": dzm["orth"],
            "note": "double-float factor and Q^T b; thin-Q WY products as Ozaki splits (7 balanced base-256 "
                    "digits) on tcgen05"}
        f3 = run_mode(0, args.steps, min(args.warmup, 3), False, f32=True)
        s_ms = f3["ms"] / args.steps
        forms["fp32"] = {
            "dtype": "f32", "value": per_step * world / (s_ms / 1e3) / 1e9, "unit": "GFLOP/s",
            "ms_per_step": s_ms, "speedup_vs_f64": ms_step / s_ms,
            "kernel_ms": {k: statistics.mean(v) for k, v in f3["ev"].items()},
            "backward_error": f3["be"], "orthogonality": f3["orth"],
            "note": "FP32 storage (A rounded to float32, R, Q, b float32) and FP32 arithmetic; "
                    "measures against the float32 A, bar 5e-5"}
        # the blocked factor step whose WY products and Gram entries run on the tensor cores
        # (64-row leaves): Ozaki splits with FP64 reflectors, bf16x3 terms with FP32 storage
        for nm, prec, f32, note in (
                ("ozaki_wy_blocked", 2, False, "mode 2 with 64-row leaves: blocked factor step, FP64 panel "
                 "reflectors, panel WY products and Gram entries as Ozaki splits on tcgen05; thin Q as ozaki_wy"),
                ("fp32_blocked", 0, True, "FP32 storage with 64-row leaves: blocked factor step, FP32 panel "
                 "reflectors, panel WY products and Gram entries as bf16x3 terms on tcgen05; thin Q as fp32")):
            r = run_mode(prec, args.steps, min(args.warmup, 3), False, f32=f32, leaf_h=64)
            r_ms = r["ms"] / args.steps
            forms[nm] = {"precision": prec, "leaf_h": 64, "dtype": "f32" if f32 else "f64+bf16x8-slice-split",
                         "value": per_step * world / (r_ms / 1e3) / 1e9, "unit": "GFLOP/s", "ms_per_step": r_ms,
                         "speedup_vs_f64": ms_step / r_ms,
                         "kernel_ms": {k: statistics.mean(v) for k, v in r["ev"].items()},
                         "backward_error": r["be"], "orthogonality": r["orth"], "note": note}
        ab_ = algorithmic_bytes(m, n)
        for nm, fm in forms.items():
            fm["roofline"] = form_roofline(nm, fl, fm["kernel_ms"], ab_, peaks, pipes)
        opts = tsqr.Opts(precision=0)

    # batched TSQR: 512 uneven matrices in one persistent launch (CUDA graph) vs a per-matrix loop
    batched = None
    if not args.no_batched and world == 1:
        batched = run_batched(tsqr, torch, dev, stream, sptr, args)

    # R alone (the paper times R alone and Q with R apart): no reflectors, T or tree factors
    r_alone = None
    if not args.no_forms and world == 1:
        r_alone = {"flops": "2mn^2 - 2n^3/3 per factorization"}
        for nm, prec, f32 in (("fp64", 0, False), ("double_float", 1, False), ("fp32", 0, True)):
            X = A.float() if f32 else A
            Rx = torch.empty((n, n), dtype=X.dtype, device=dev)
            o = tsqr.Opts(precision=prec, r_only=1)
            code = tsqr.TSQR_F32 if f32 else tsqr.TSQR_F64
            nb = tsqr.tsqr_workspace_size(code, m, n, o)
            wk = torch.empty(nb, dtype=torch.uint8, device=dev)
            ts = []
            for it in range(1 + max(2, min(args.steps, 5))):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h = tsqr.tsqr_factor(code, tsqr.TSQR_ROW_MAJOR, m, n, X.data_ptr(), n, Rx.data_ptr(), n,
                                     wk.data_ptr(), nb, o, sptr)
                e1.record(stream)
                tsqr.tsqr_destroy(h)
                torch.cuda.synchronize()
                if it:
                    ts.append(e0.elapsed_time(e1))
            t = statistics.mean(ts)
            r_alone[nm] = {"factor_ms": t, "value": fl["factor"] / (t / 1e3) / 1e9, "unit": "GFLOP/s",
                           "workspace_bytes": nb}
            del X, Rx, wk
        torch.cuda.empty_cache()

    # context, not a target: the vendor library's QR of the same matrix (torch.linalg.qr, cuSOLVER)
    library = None
    if not args.no_forms and world == 1:
        library = {"what": "torch.linalg.qr (cuSOLVER geqrf + orgqr) on the same A, explicit Q and R"}
        for nm, X in (("fp64", A), ("fp32", A.float())):
            torch.linalg.qr(X)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(2):
                Qc, Rc = torch.linalg.qr(X)
            e1.record(stream)
            torch.cuda.synchronize()
            c_ms = e0.elapsed_time(e1) / 2
            fl2 = flops(m, n)
            library[nm] = {"ms": c_ms, "value": (fl2["factor"] + fl2["form_q"]) / (c_ms / 1e3) / 1e9,
                           "unit": "GFLOP/s (factor + thin Q)"}
            del Qc, Rc, X
        torch.cuda.empty_cache()

    # Q^T B and Q B with 64 columns on the benchmark's matrix: the WY products of the apply on the
    # FP64 / FP32 pipes (mode 0) or on the tensor cores (modes 2 and 3, FP32 storage)
    apply_wide = None
    if (not args.no_forms or args.apply_wide) and world == 1:
        apply_wide = run_apply_wide(tsqr, torch, dev, stream, sptr, A, m, n)

    shapes = None
    if not args.no_shapes and world == 1:
        shapes = run_shapes(tsqr, torch, dev, stream, sptr, m)

    tree_levels = None
    if not args.no_shapes and world == 1:
        tree_levels = run_tree_levels(tsqr, torch, dev, stream, sptr)

    conditioning = None
    if not args.no_conditioning and world == 1:
        conditioning = run_conditioning(tsqr, torch, dev, stream, sptr, m, n)

    autograd = None
    if not args.no_autograd and world == 1:
        autograd = run_autograd(tsqr, torch, dev, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rows = args.cpu_rows
        gf, dt, _ = cpu_oracle_sample(A_h, rows)
        gfo, dto, thr = cpu_oracle_sample(A_h, rows, openmp=True)
        cpu = {"value": gf, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
               "sample": "oracle QR, thin Q and Q^T b of the first %d rows of the same matrix (%.1f s)" % (rows, dt),
               "openmp": {"value": gfo, "unit": "GFLOP/s", "cores": thr, "seconds": dto,
                          "what": "the same oracle source built with -fopenmp (its reflector applications run "
                                  "column-parallel; results bitwise the serial build's), same sample"},
               "host": host_cpu(), "library_cpu": cpu_library_sample(torch, A_h, rows)}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32" if args.fp32 else {0: "f64", 1: "f32x2", 2: "f64", 3: "f32x2"}[args.precision], "data": "synthetic",
               "config": main_config(m, n, args.precision, world),
               "backward_error": be, "orthogonality": orth,
               "kernel_ms": {"factor": f_ms, "form_q": q_ms, "apply_qt": a_ms},
               "roofline": roofline, "precision_forms": forms, "apply_wide": apply_wide, "batched": batched,
               "shapes": shapes, "conditioning": conditioning, "tree_levels": tree_levels,
               "autograd": autograd, "r_alone": r_alone, "library_context": library, "cpu_baseline": cpu,
               "e2e": e2e,
               "gpu_launches": main_mode["launches"] * args.steps, "clocks": clocks}
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
