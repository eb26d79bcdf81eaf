"""Benchmark: spaND factor + s-step GMRES solve of the DG Newton-step system.

Workload (default, the largest single-GPU configuration): p=3 modal DG Jacobian
of 2D Euler on a seeded 256 x 128 NACA O-grid (K=32,768, N=2,097,152, blocks
64 x 64, A = 5.35 GB in FP64), M=0.8 with +-10% perturbations, spaND eps=1e-3,
s-step GMRES s=8, restart 80, tol 1e-8.  One step = spand_factor +
sstep_gmres_solve to a true FP64 relative residual <= 1e-8, inputs resident in
HBM (A and the factors are larger than the L2; the L2 is also flushed between
timed steps).  The headline form is the mixed one (FP32 / TF32 factor and
apply, FP64 SpMV / Gram / CholQR / Hessenberg); the FP64 form is timed beside it
for the speedup.  The 64 x 32 p=2 workload (N=73,728) is measured as a
secondary sub-object (`secondary_C2`), with the pseudo-time continuation and the
Krylov stress setting.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--config C2|C3|C5]

--impl reference times the CPU oracle (NumPy/SciPy) on a bounded sample of the
same workload (a p=3 32 x 16 O-grid with the same flow and solver settings),
scaled to the full workload by its number of unknowns (spaND factor and solve
cost grow linearly with N in 2D, Sec. 2.2.1).
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
sys.path.insert(0, ROOT)

METRIC = "spaND factor+s-step GMRES time to 1e-8 rel residual; mixed vs FP64 speedup"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# FP64 arithmetic peak of a GB300 (nominal, the profiling recipe's table: the
# FP64 rate is a small fraction of the FP32 one on this part).  The FP64 block
# SpMV, Gram reductions and block updates are bound by it, not by HBM.
FP64_TFLOPS_NOMINAL = 1.25


def dual_bound(entry, flops, hbm_frac):
    """Add the FP64 arithmetic view of an FP64 kernel and pick as `bound` the
    roof it is closer to (the binding one)."""
    ms = entry["ms_per_launch"]
    tf = flops / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
    entry["fp64_tflops"] = tf
    entry["fp64_frac"] = tf / FP64_TFLOPS_NOMINAL
    entry["fp64_peak_kind"] = "nominal FP64 1.25 TFLOP/s (profiling recipe table)"
    entry["flops_per_launch"] = flops
    if entry["fp64_frac"] > hbm_frac:
        entry.update(bound="alu", achieved=tf, peak=FP64_TFLOPS_NOMINAL, unit="TFLOP/s", frac=entry["fp64_frac"],
                     peak_kind=entry["fp64_peak_kind"], hbm_frac=hbm_frac)
    return entry
# the oracle sample behind the CPU baseline and the reference arm: the same
# flow and solver settings on a small grid of the same degree
CPU_SAMPLE_GRID = (32, 16)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--config", default="C3")
    return ap.parse_args()


def workload(cname):
    from synth import get_config, modal_state, naca_ogrid
    c = get_config(cname)
    X = naca_ogrid(c.n_theta, c.n_r, c.seed)
    u = modal_state(X, c.p, c.mach, c.alpha_deg, c.amp, c.seed)
    return c, X, u


def config_json(c):
    """The workload as both arms print it (identical dicts)."""
    return {"workload": f"DG Euler Jacobian p={c.p} O-grid {c.n_theta}x{c.n_r} (K={c.K}, N={c.N}), "
                        f"M={c.mach}, +-{int(round(100 * c.amp))}% perturbation, spaND eps={c.eps}, "
                        f"s-step GMRES s={c.s} restart={c.restart} tol={c.tol}",
            "N": c.N, "block": c.B, "eps": c.eps, "s": c.s, "restart": c.restart, "tol": c.tol,
            "l2": "inputs larger than L2 when N > 1e6 (A and the factors are GBs); "
                  "also flushed between timed steps (256 MB write)"}


def oracle_sample(c, reps, warm=0):
    """The oracle (factor + s-step GMRES) on the CPU sample of workload c: the
    same p, flow and solver settings on a CPU_SAMPLE_GRID O-grid.  Returns
    (seconds per sample, the sample's N, stats of the last solve)."""
    from oracle import dg, spand
    from oracle.gmres import sstep_gmres
    from synth import modal_state, naca_ogrid
    nt, nr = CPU_SAMPLE_GRID
    cs = c.with_(n_theta=min(nt, c.n_theta), n_r=min(nr, c.n_r))
    X = naca_ogrid(cs.n_theta, cs.n_r, cs.seed)
    u = modal_state(X, cs.p, cs.mach, cs.alpha_deg, cs.amp, cs.seed)
    rhs, bsr, _ = dg.assemble(X, cs.p, u, cs.mach, cs.alpha_deg, cs.cfl)
    A = dg.bsr_to_scipy(*bsr).tocsr()
    times, st = [], None
    for k in range(warm + reps):
        t0 = time.perf_counter()
        F = spand.factor(bsr, cs.n_theta, cs.n_r, cs.nd_depth, cs.eps)
        _, st = sstep_gmres(lambda v: A @ v, lambda v: spand.apply(F, v), rhs, s=cs.s, restart=cs.restart,
                            tol=cs.tol, max_iters=cs.max_iters)
        if k >= warm:
            times.append(time.perf_counter() - t0)
    return times, cs, st


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, idx=0):
        self.idx = idx
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for n, v in zip(names, s[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return d, "measured"
        except Exception:
            pass
    return dict(PEAKS_FALLBACK), "fallback"


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise max of per-rank values (the slowest rank's times) by one
    all_reduce; the values themselves when there is no process group."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def run_reference(args):
    """CPU oracle arm: each step is one oracle factor + s-step GMRES solve of the
    bounded sample (same p, flow and solver settings on a small O-grid),
    reported in the workload's unit (ms per solve of the full workload) by
    scaling with the ratio of unknowns; W untimed warm-up samples first."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from synth import get_config
    c = get_config(args.config)
    times, cs, st = oracle_sample(c, max(1, args.steps), warm=max(0, args.warmup))
    scale = c.N / cs.N
    ms = 1e3 * statistics.mean(times) * scale
    cores = os.cpu_count()
    sample = (f"oracle factor+solve of a p={cs.p} {cs.n_theta}x{cs.n_r} O-grid (N={cs.N}) with the workload's "
              f"flow and solver settings, x {scale:.1f} (ratio of unknowns; spaND is O(N) in 2D)")
    out = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus, "steps": len(times),
           "warmup": max(0, args.warmup), "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": config_json(c),
           "cpu_baseline": {"value": ms, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "sample_s_per_step": statistics.mean(times), "sample_true_relres": float(st.true_relres),
           "sample_iters": st.iters}
    print(json.dumps(out))
    return 0


def run_batch(args):
    """Many independent systems (grids, degrees, flow conditions drawn per
    system): batched mixed factorization + batched s-step GMRES, against the
    same systems solved one at a time in FP64 and in mixed precision."""
    import torch
    from synth.configs import batch_configs
    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__ as g
    g.build()
    import paper_2101_01763_gb300 as sg
    from synth import modal_state, naca_ogrid
    cs = batch_configs(24)
    sys_ = []
    for c in cs:
        X = naca_ogrid(c.n_theta, c.n_r, c.seed)
        u = modal_state(X, c.p, c.mach, c.alpha_deg, c.amp, c.seed)
        rhs, A, _ = sg.assemble(torch.as_tensor(X, device=dev), c.p, torch.as_tensor(u, device=dev), c.mach,
                                c.alpha_deg, c.cfl)
        sys_.append((c, A, rhs, sg.Plan(c.n_theta, c.n_r, A.B, c.nd_depth)))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    c0 = cs[0]

    # systems are factored in groups of at most ~3M unknowns (the union of a
    # level's clusters, its W matrices and the factors of a group stay well
    # inside HBM); a group's factors are released before the next group
    groups, cur, tot = [], [], 0
    for q, (c, A, b, p) in enumerate(sys_):
        if cur and tot + c.N > 3_000_000:
            groups.append(cur)
            cur, tot = [], 0
        cur.append(q)
        tot += c.N
    if cur:
        groups.append(cur)

    grp_ms = [0.0] * len(groups)

    def batched():
        xs, st, status = [None] * len(sys_), [None] * len(sys_), [None] * len(sys_)
        for gi, grp in enumerate(groups):
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            Fb = sg.factor_batched([sys_[q][3] for q in grp], [sys_[q][1] for q in grp], c0.eps, "mixed")
            x_g, st_g, s_g = sg.sstep_gmres_batched([sys_[q][1] for q in grp], Fb, [sys_[q][2] for q in grp],
                                                    s=c0.s, restart=c0.restart, tol=c0.tol, max_iters=c0.max_iters)
            g1.record(stream)
            torch.cuda.synchronize()
            grp_ms[gi] = g0.elapsed_time(g1)
            for f in Fb:
                f.close()
            for k, q in enumerate(grp):
                xs[q], st[q], status[q] = x_g[k], st_g[k], s_g[k]
        return [], xs, st, status

    sys_ms = {"mixed": [0.0] * len(sys_), "fp64": [0.0] * len(sys_)}

    def single(prec):
        out = []
        for q, (c, A, b, plan) in enumerate(sys_):
            q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            F = sg.Factor(plan, A, c.eps, prec)
            x, st = sg.sstep_gmres(A, F, b, s=c.s, restart=c.restart, tol=c.tol, max_iters=c.max_iters)
            q1.record(stream)
            torch.cuda.synchronize()
            sys_ms[prec][q] = q0.elapsed_time(q1)
            out.append((x, st))
            F.close()
        return out

    def timed(fn, steps, warm):
        for _ in range(warm):
            r = fn()
            if isinstance(r, tuple):
                for f in r[0]:
                    f.close()
        ts = []
        res = None
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            if isinstance(res, tuple):
                for f in res[0]:
                    f.close()
        return statistics.mean(ts), res

    steps, warm = max(1, args.steps), max(1, min(args.warmup, 3))
    with Clocks(local) as clk:
        t_b, (_, xs, st_b, status) = timed(batched, steps, warm)
    t_m, res_m = timed(lambda: single("mixed"), 1, 1)
    t_64, res_64 = timed(lambda: single("fp64"), 1, 1)
    rel = []
    for (c, A, b, _), x in zip(sys_, xs):
        r = sg.spmv(A, x) - b
        rel.append((torch.linalg.norm(r) / torch.linalg.norm(b)).item())
    if rank != 0:
        return 0
    n = len(cs)
    out = {"metric": "independent DG Newton-step systems solved per second (spaND factor + s-step GMRES, "
                     "batched mixed precision)",
           "value": world * n * 1e3 / t_b, "unit": "systems/s", "n_gpus": world, "steps": steps, "warmup": warm,
           "ms_per_step": t_b, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": f"{n} systems: O-grids in {{32x16, 64x32, 96x48, 192x96}}, p in {{1,2,3}}, "
                                  f"M in [0.3,0.8], alpha in [0,4] deg (seeds 2101_0500+i), eps={c0.eps}, "
                                  f"s={c0.s}, restart={c0.restart}, tol={c0.tol}",
                      "total_N": sum(c.N for c in cs), "groups": [len(g) for g in groups],
                      "l2": "flushed between timed steps (256 MB write)"},
           "ms_per_system_batched": t_b / n, "ms_one_at_a_time_mixed": t_m, "ms_one_at_a_time_fp64": t_64,
           "speedup_vs_one_at_a_time_fp64": t_64 / t_b, "speedup_vs_one_at_a_time_mixed": t_m / t_b,
           "max_true_relres": max(rel), "all_converged": all(v == 0 for v in status),
           "iters": [s["iters"] for s in st_b], "clocks": clk.summary(),
           "per_group": [{"systems": len(grp), "N": [cs[q].N for q in grp], "batched_ms": grp_ms[gi],
                          "one_at_a_time_mixed_ms": sum(sys_ms["mixed"][q] for q in grp),
                          "one_at_a_time_fp64_ms": sum(sys_ms["fp64"][q] for q in grp)}
                         for gi, grp in enumerate(groups)]}
    print(json.dumps(out))
    return 0


class Workload:
    """One configuration on the device: seeded grid and state, assembled A and
    b (device), the ND plan."""

    def __init__(self, sg, torch, dev, name):
        self.c, X, u = workload(name)
        self.Xd = torch.as_tensor(X, device=dev)
        self.ud = torch.as_tensor(u, device=dev)
        c = self.c
        self.rhs, self.A, self.dtau = sg.assemble(self.Xd, c.p, self.ud, c.mach, c.alpha_deg, c.cfl)
        self.plan = sg.Plan(c.n_theta, c.n_r, c.B, c.nd_depth)
        self.X, self.u = X, u


def timed_steps(sg, torch, W, prec, steps, warmup, flush, stream, barrier):
    """W warm-up then `steps` timed factor + solve steps (CUDA events on the
    launching stream, L2 flushed before each).  Returns the per-step (factor ms,
    solve ms), the last step's (factor stats, solve stats, x) and the library's
    kernel launches in the timed steps."""
    c = W.c

    def one():
        F = sg.Factor(W.plan, W.A, c.eps, prec)
        x, st = sg.sstep_gmres(W.A, F, W.rhs, s=c.s, restart=c.restart, tol=c.tol, max_iters=c.max_iters)
        return F, x, st

    for _ in range(warmup):
        F, x, st = one()
        F.close()
    ev, last = [], None
    barrier()
    n0 = sg.kernel_launches()
    for _ in range(steps):
        flush.fill_(1.0)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        F = sg.Factor(W.plan, W.A, c.eps, prec)
        e1.record(stream)
        x, st = sg.sstep_gmres(W.A, F, W.rhs, s=c.s, restart=c.restart, tol=c.tol, max_iters=c.max_iters)
        e2.record(stream)
        torch.cuda.synchronize()
        ev.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
        last = (F.stats(), st, x)
        F.close()
    barrier()
    return ev, last, sg.kernel_launches() - n0


def true_relres(sg, torch, W, x):
    r = sg.spmv(W.A, x)
    return (torch.linalg.norm(r - W.rhs) / torch.linalg.norm(W.rhs)).item()


def rooflines(sg, torch, W, fst, flush, stream, peaks_):
    """Live rooflines of the kernels of one workload: RRQR (from the last timed
    factorization's events), elimination GEMMs, the apply sweeps, the block SpMV."""
    pk, pk_kind = peaks_
    c = W.c
    hbm = float(pk.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    # the GEMMs run inside a seconds-long factorization: the sustained bf16 figure
    bf16 = float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"])))
    tf32_peak = bf16 * (1.1 / 2.25)          # nominal TF32 : BF16 dense ratio
    # rank-revealing QR of the sparsification (k_qrcp_stream); one "launch" = the
    # RRQR phase of one level (its kernels between two events on the factor's
    # stream).  Bound by the traffic of the live columns: the kernel counts the
    # bytes its column passes move (each live column read and written once per
    # pivot step).  The method's own work, 4 (n-k)(c-k) flops per pivot step
    # (reflector dot products and update over every column), is reported beside.
    nl = max(1, fst["rrqr_launches"])
    rr_ms = fst["t_rrqr_ms"] / nl
    rr_bytes = fst["rrqr_stream_bytes"] / nl
    rr_ach = rr_bytes / (rr_ms * 1e-3) / 1e9 if rr_ms > 0 else 0.0
    rr_flops = 4.0 * (fst["rrqr_bytes"] / 8.0) / nl
    gm_ms = fst["t_elim_gemm_ms"] / max(1, fst["elim_gemm_launches"])
    gm_fl = fst["elim_gemm_flops"] / max(1, fst["elim_gemm_launches"])
    gm_ach = gm_fl / (gm_ms * 1e-3) / 1e12 if gm_ms > 0 else 0.0
    F = sg.Factor(W.plan, W.A, c.eps, "mixed")
    z = torch.empty_like(W.rhs)
    for _ in range(3):
        F.apply(W.rhs, out=z)
    napp = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(napp):
        F.apply(W.rhs, out=z)
    e1.record(stream)
    torch.cuda.synchronize()
    t_apply = e0.elapsed_time(e1) / napp
    fb = F.stats()["factor_bytes"]
    F.close()
    app_ach = fb / (t_apply * 1e-3) / 1e9
    # block SpMV (FP64): A's blocks and two vectors per launch, L2 flushed before each
    y = torch.empty_like(W.rhs)
    sp_ms = []
    for it in range(13):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sg.spmv(W.A, W.rhs, out=y)
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= 3:
            sp_ms.append(e0.elapsed_time(e1))
    t_spmv = statistics.mean(sp_ms)
    sp_bytes = W.A.nnzb * W.A.B * W.A.B * 8 + 2 * W.A.K * W.A.B * 8
    sp_ach = sp_bytes / (t_spmv * 1e-3) / 1e9
    rr = {"kernel": "k_qrcp_stream (column-pivoted Householder QR of the interface sparsification, W streamed "
                    "from L2/HBM; one launch = the RRQR phase of one level)",
          "bound": "hbm", "achieved": rr_ach, "peak": hbm, "unit": "GB/s", "frac": rr_ach / hbm, "traffic": None,
          "peak_kind": f"{pk_kind} hbm_gbs", "bytes_per_launch": rr_bytes, "ms_per_launch": rr_ms,
          "bytes_rule": "2 (n-k) m_k x 4 per pivot step k, m_k = live columns (counted by the kernel)",
          "method_flops_per_launch": rr_flops,
          "method_tflops": rr_flops / (rr_ms * 1e-3) / 1e12 if rr_ms > 0 else 0.0,
          "method_flops_rule": "4 (n-k)(c-k) per pivot step k over every column"}
    gm = {"kernel": "k_gemm_umma / k_gemm_tc (elimination Y, X, Schur products; 3xTF32, FP32 accumulation)",
          "bound": "tensor", "achieved": gm_ach, "peak": tf32_peak, "unit": "TFLOP/s", "frac": gm_ach / tf32_peak,
          "traffic": None, "peak_kind": f"{pk_kind} sustained bf16 x nominal tf32/bf16 ratio (1.1/2.25)",
          "flops_per_launch": gm_fl, "ms_per_launch": gm_ms, "flops_rule": "useful flops: 2 m n k per full product (Schur), m n k per triangular-times-dense "
                       "product (Y = L^-1 P^T A_sn, X = A_ns U^-1)"}
    more = [
        {"kernel": "spand_apply (k_gemv sweeps, FP32 factors)", "bound": "hbm", "achieved": app_ach,
         "peak": hbm, "unit": "GB/s", "frac": app_ach / hbm, "peak_kind": f"{pk_kind} hbm_gbs",
         "bytes_per_launch": fb, "ms_per_launch": t_apply},
        dual_bound({"kernel": "k_bsr_spmv (FP64 block SpMV, L2 flushed before each launch)", "bound": "hbm",
                    "achieved": sp_ach, "peak": hbm, "unit": "GB/s", "frac": sp_ach / hbm,
                    "peak_kind": f"{pk_kind} hbm_gbs", "bytes_per_launch": sp_bytes, "ms_per_launch": t_spmv},
                   2.0 * W.A.nnzb * W.A.B * W.A.B, sp_ach / hbm)]
    # the headline roofline is the kernel family that takes the most factor time
    if fst["t_elim_gemm_ms"] >= fst["t_rrqr_ms"]:
        return gm, [rr] + more
    return rr, [gm] + more
    return rr, more


def gram_rooflines(sg, torch, W, hbm, pk_kind):
    """The single-reduction kernels of Algorithm 2 at the workload's N, s and
    restart: one full unpreconditioned s-step cycle (restart columns, so every
    s-block runs its block Gram reduction and its CGS2 / CholQR2 updates), timed
    per launch by the solver's own events."""
    c = W.c
    kw = dict(s=c.s, restart=c.restart, tol=0.0, max_iters=c.restart)
    sg.sstep_gmres(W.A, None, W.rhs, **kw)
    _, st = sg.sstep_gmres(W.A, None, W.rhs, **kw)
    out = []
    # flops: the Gram G = Z^T Y is 2 nz ny N per reduction; a block update X = Y S^-1 - Z C is
    # 2 (ny + nz) s N.  The byte counts above fix nz + ny and ny + nz + s per launch, and
    # ny = 2s (Gram: Y = [P, V]) or s (update), so the flop counts follow from them.
    s_ = c.s
    for name, t, b, n, rule, kind in (
            ("k_gram_partial + k_gram_reduce (block Gram G = [Q_f, P, V]^T [P, V], FP64)", st["t_gram_ms"],
             st["gram_bytes"], st["gram_calls"], "(nz + ny) N 8 bytes per reduction", 0),
            ("k_block_update (CGS2 / CholQR2 block updates X = Y S^-1 - Z C, FP64)", st["t_bupd_ms"],
             st["bupd_bytes"], st["bupd_calls"], "(ny + nz + s) N 8 bytes per update", 1)):
        ms = t / max(1, n)
        bl = b / max(1, n)
        ach = bl / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        vec = bl / (8.0 * c.N)                 # vectors read per launch
        if kind == 0:
            ny = min(2 * s_, vec / 2)
            fl = 2.0 * (vec - ny) * ny * c.N
        else:
            fl = 2.0 * (vec - s_) * s_ * c.N
        out.append(dual_bound({"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                               "frac": ach / hbm, "peak_kind": f"{pk_kind} hbm_gbs", "bytes_per_launch": bl,
                               "ms_per_launch": ms, "launches": n, "bytes_rule": rule,
                               "setting": f"one unpreconditioned s-step cycle, s={c.s}, restart={c.restart}, N={c.N}"},
                              fl, ach / hbm))
    return out


def march_and_stress(sg, torch, W, stream):
    """The pseudo-time continuation around the step (Eq. 9 CFL ramp, plan reused,
    A re-assembled and re-factored at every step) and the Krylov stress setting
    (eps = 1e-1, tolerance 1e-10, at most 100 steps): Algorithm 1 beside
    Algorithm 2 with their per-phase stream times."""
    c = W.c
    mopts = dict(cfl0=c.cfl, cfl_inf=1e6, rtol=0.0, eps=c.eps, precision="mixed", s=c.s, restart=c.restart,
                 tol=c.tol, max_iters=c.max_iters)
    try:
        sg.march(W.Xd, c.p, W.ud, c.mach, c.alpha_deg, W.plan, max_steps=1, **mopts)
        nm = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        _, hm = sg.march(W.Xd, c.p, W.ud, c.mach, c.alpha_deg, W.plan, max_steps=nm, **mopts)
        e1.record(stream)
        torch.cuda.synchronize()
        tm = e0.elapsed_time(e1)
        march = {"pseudo_time_steps": hm["steps"], "ms": tm, "ms_per_pseudo_time_step": tm / max(1, hm["steps"]),
                 "per_step": "assemble + ||R|| + spand_factor + s-step GMRES + update (and the final assembly)",
                 "cfl0": c.cfl, "cfl_inf": 1e6, "res_norm": [float(v) for v in hm["res"]],
                 "cfl": [float(v) for v in hm["cfl"]], "gmres_iters": [int(v) for v in hm["gmres_iters"]]}
    except Exception as ex:   # reported, never fatal to the headline line
        march = {"error": str(ex)}
    krylov = None
    try:
        Fs = sg.Factor(W.plan, W.A, 0.1, "mixed")
        krylov = {"eps": 0.1, "tol": 1e-10, "max_iters": 100, "restart": 60, "s": c.s, "factor": "mixed"}
        for name, call in (("gmres_mgs", lambda: sg.gmres(W.A, Fs, W.rhs, restart=60, tol=1e-10, max_iters=100)),
                           ("sstep_gmres", lambda: sg.sstep_gmres(W.A, Fs, W.rhs, s=c.s, restart=60, tol=1e-10,
                                                                  max_iters=100))):
            call()
            n0 = sg.kernel_launches()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            _, kst = call()
            e1.record(stream)
            torch.cuda.synchronize()
            krylov[name] = {"ms": e0.elapsed_time(e1), "iters": kst["iters"], "converged": kst["converged"],
                            "true_relres": kst["true_relres"], "reductions": kst["reductions"],
                            "launches": sg.kernel_launches() - n0,
                            "phase_ms": {"spmv": kst["t_spmv_ms"], "apply": kst["t_apply_ms"],
                                         "orth": kst["t_orth_ms"], "other": kst["t_small_ms"]},
                            "gram": {"calls": kst["gram_calls"], "ms": kst["t_gram_ms"], "bytes": kst["gram_bytes"],
                                     "gbs": kst["gram_bytes"] / (kst["t_gram_ms"] * 1e-3) / 1e9
                                     if kst["t_gram_ms"] > 0 else None}}
        Fs.close()
    except Exception as ex:
        krylov = {"error": str(ex)}
    return march, krylov


def e2e_steps(sg, torch, W, steps, warmup, flush):
    """The metric end to end through the public API: every step copies A's values
    and pattern and b from pinned host memory, factors, solves and reads x back."""
    c, A = W.c, W.A
    h_val = A.val.cpu().pin_memory()
    h_rp = A.row_ptr.cpu().pin_memory()
    h_col = A.col.cpu().pin_memory()
    h_b = W.rhs.cpu().pin_memory()
    h_x = torch.empty_like(h_b).pin_memory()
    d_val = torch.empty_like(A.val)
    d_rp = torch.empty_like(A.row_ptr)
    d_col = torch.empty_like(A.col)
    d_b = torch.empty_like(W.rhs)
    A2 = sg.BSR(A.K, A.B, d_rp, d_col, d_val)
    ts = []
    for it in range(warmup + steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d_val.copy_(h_val, non_blocking=True)
        d_rp.copy_(h_rp, non_blocking=True)
        d_col.copy_(h_col, non_blocking=True)
        d_b.copy_(h_b, non_blocking=True)
        F2 = sg.Factor(W.plan, A2, c.eps, "mixed")
        x2, _ = sg.sstep_gmres(A2, F2, d_b, s=c.s, restart=c.restart, tol=c.tol, max_iters=c.max_iters)
        h_x.copy_(x2, non_blocking=True)
        torch.cuda.synchronize()
        if it >= warmup:
            ts.append(time.perf_counter() - t0)
        F2.close()
    del d_val, h_val
    bi = A.nnzb * A.B * A.B * 8 + (A.K + 1) * 4 + A.nnzb * 4 + h_b.numel() * 8
    bo = h_x.numel() * 8
    return 1e3 * statistics.mean(ts), bi, bo


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "C5":
        return run_batch(args)
    import numpy as np
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__ as g
    g.build()
    import paper_2101_01763_gb300 as sg
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    W = Workload(sg, torch, dev, args.config)
    c = W.c
    big = c.N > 1_000_000
    # ---- headline: mixed form, exactly K timed steps after W warm-up steps
    with Clocks(local) as clk:
        ev_mx, (fst_mx, gst_mx, x_mx), launches_mx = timed_steps(sg, torch, W, "mixed", args.steps, args.warmup,
                                                                 flush, stream, barrier)
    relres = true_relres(sg, torch, W, x_mx)
    # ---- FP64 form beside it (FP64-ALU bound factorization: fewer steps at the large size)
    k64, w64 = (1, 1) if big else (max(2, min(args.steps, 4)), max(1, min(args.warmup, 2)))
    ev_64, (fst_64, gst_64, x_64), _ = timed_steps(sg, torch, W, "fp64", k64, w64, flush, stream, barrier)
    relres64 = true_relres(sg, torch, W, x_64)
    t_mx = statistics.mean(a + b for a, b in ev_mx)
    t_64 = statistics.mean(a + b for a, b in ev_64)
    clk_sum = clk.summary()
    rr, more = rooflines(sg, torch, W, fst_mx, flush, stream, peaks())
    pk, pk_kind = peaks()
    more += gram_rooflines(sg, torch, W, float(pk.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])), pk_kind)
    # ---- end to end through the C ABI with host buffers (pinned), copies inside
    ke, we = (min(args.steps, 3), 1) if big else (args.steps, args.warmup)
    t_e2e, bi, bo = e2e_steps(sg, torch, W, ke, we, flush)
    sec = None
    if args.config == "C3":
        # ---- the 64 x 32 p=2 workload as a secondary sub-object
        W2 = Workload(sg, torch, dev, "C2")
        k2 = max(3, min(args.steps, 10))
        ev2, (fst2, gst2, x2), l2 = timed_steps(sg, torch, W2, "mixed", k2, 3, flush, stream, barrier)
        ev2_64, (_, g2_64, _), _ = timed_steps(sg, torch, W2, "fp64", 3, 1, flush, stream, barrier)
        rr2, more2 = rooflines(sg, torch, W2, fst2, flush, stream, peaks())
        march2, krylov2 = march_and_stress(sg, torch, W2, stream)
        t2 = statistics.mean(a + b for a, b in ev2)
        t2_64 = statistics.mean(a + b for a, b in ev2_64)
        sec = {"config": config_json(W2.c), "ms_per_step_mixed": t2, "ms_per_step_fp64": t2_64,
               "speedup_mixed_vs_fp64": t2_64 / t2, "steps": k2, "fp64_steps": 3,
               "factor_ms": statistics.mean(a for a, _ in ev2), "solve_ms": statistics.mean(b for _, b in ev2),
               "gmres_iters_mixed": gst2["iters"], "gmres_iters_fp64": g2_64["iters"],
               "reductions_mixed": gst2["reductions"], "true_relres_mixed": true_relres(sg, torch, W2, x2),
               "gpu_launches_per_step": l2 / k2, "rrqr_ms_per_level": fst2["t_rrqr_level_ms"],
               "ranks_per_level": fst2["sum_r"], "roofline": rr2, "roofline_more": more2,
               "pseudo_time_march": march2, "krylov_stress": krylov2}
        del W2

    # ---- max over ranks
    t_mx, t_64, t_e2e = max_over_ranks([t_mx, t_64, t_e2e], dist, dev)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # ---- CPU baseline: the oracle on a bounded sample of the workload, scaled
    cpu = None
    if world == 1 and os.environ.get("BENCH_SKIP_CPU", "0") != "1":
        times, cs, st = oracle_sample(c, 3 if big else 1)
        scale = c.N / cs.N
        cpu = {"value": 1e3 * statistics.mean(times) * scale, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{len(times)} oracle factor+solve(s) of a p={cs.p} {cs.n_theta}x{cs.n_r} O-grid "
                         f"(N={cs.N}) with the workload's flow and solver settings, mean x {scale:.1f} "
                         f"(ratio of unknowns; spaND is O(N) in 2D)",
               "sample_s": statistics.mean(times), "sample_true_relres": float(st.true_relres)}
        if not big:
            from oracle import dg, spand
            from oracle.gmres import sstep_gmres
            rhs_o, bsr, _ = dg.assemble(W.X, c.p, W.u, c.mach, c.alpha_deg, c.cfl)
            So = dg.bsr_to_scipy(*bsr).tocsr()
            Fo = spand.factor(bsr, c.n_theta, c.n_r, c.nd_depth, c.eps)
            xo, _ = sstep_gmres(lambda v: So @ v, lambda v: spand.apply(Fo, v), rhs_o, s=c.s, restart=c.restart,
                                tol=c.tol, max_iters=c.max_iters)
            cpu["mixed_solution_rel_err_vs_oracle"] = float(np.linalg.norm(x_mx.cpu().numpy() - xo)
                                                            / np.linalg.norm(xo))
    out = {
        "metric": METRIC, "value": t_mx, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_mx, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": config_json(c),
        "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
        "form": "mixed (FP32/TF32 factor+apply, FP64 outer)",
        "fp64_ms_per_step": t_64, "fp64_steps": k64, "fp64_warmup": w64, "speedup_mixed_vs_fp64": t_64 / t_mx,
        "factor_ms": statistics.mean(a for a, _ in ev_mx), "solve_ms": statistics.mean(b for _, b in ev_mx),
        "fp64_factor_ms": statistics.mean(a for a, _ in ev_64), "fp64_solve_ms": statistics.mean(b for _, b in ev_64),
        "gmres_iters_mixed": gst_mx["iters"], "gmres_iters_fp64": gst_64["iters"],
        "reductions_mixed": gst_mx["reductions"], "reductions_fp64": gst_64["reductions"],
        "sstep_blocks_ran": gst_mx["reductions"] > 0,
        "true_relres_mixed": relres, "true_relres_fp64": relres64,
        "mixed_vs_fp64_solution_rel_diff": (torch.linalg.norm(x_mx - x_64) / torch.linalg.norm(x_64)).item(),
        "factor_host_ms": fst_mx["t_host_ms"], "factor_gpu_wait_ms": fst_mx["t_wait_ms"],
        "factor_host_phase_ms": fst_mx["t_host_phase_ms"],
        "rrqr_ms_per_level": fst_mx["t_rrqr_level_ms"], "rrqr_forms_per_level": fst_mx["rrqr_form_count"],
        "ranks_per_level": fst_mx["sum_r"], "max_rank_per_level": fst_mx["max_r"],
        "solves_per_s": world * 1e3 / t_mx,
        "e2e": {"value": t_e2e, "unit": "ms", "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
                "steps": ke, "warmup": we},
        "gpu_launches": launches_mx,
        "gpu_launches_per_step": launches_mx / max(1, args.steps),
        "roofline": rr,
        "roofline_more": more,
        "secondary_C2": sec,
        "clocks": clk_sum,
        "cpu_baseline": cpu,
    }
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
