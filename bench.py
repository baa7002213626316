"""Benchmark of the two-site DMRG hot path on GB300 (one JSON line on stdout).

Workload: L=30 orbitals, N=30 electrons, 2S_z=0, D=1024, seeded random
integrals (stand-in for the FeMoco integrals), two-site position at the
mid-chain cut (orbitals 14, 15).  One step = one full DMRG iteration of
Sec. II.B: environments resident, enlargement of both blocks, Davidson with
H_eff products to convergence, truncation to D, renormalisation, next start
vector, and (offload on) the asynchronous pack of the new environment into
pinned host RAM (Sec. III.A/B.4).  Steps alternate between the positions
14 (moving right) and 15 (moving left), so every step rebuilds and saves one
environment.

metric: H_eff psi useful TFLOP/s = useful flops of the H_eff products in the
timed steps (2*m*k*n over the non-zero sector GEMMs, counted once) divided
by the device time of those steps (CUDA events on the library's compute
stream).  e2e: the same steps through the public API with the two-site
vector uploaded from pinned host memory before and read back after each
step.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # the smallest configuration (the oracle runs it in seconds): like-for-like pair with --impl reference
    "l10_d256": dict(L=10, N=10, tsz=0, D=256, seed=1001, b=4),
    "l30_d1024": dict(L=30, N=30, tsz=0, D=1024, seed=1002, b=14),
    # the mixed-precision configuration: 122 GB of FP64 enlarged operators at the
    # mid-chain position, run in the low-memory mode of the mixed form
    "l54_d2048": dict(L=54, N=54, tsz=0, D=2048, seed=1003, b=26),
    # a few-GB case of the same kernels, for profiler captures
    "small": dict(L=16, N=16, tsz=0, D=512, seed=1002, b=7),
}
DEFAULT_WORKLOAD = "l30_d1024"
METRIC = "H_eff psi useful TFLOP/s over whole two-site DMRG steps (mixed BF16x3 form, |dE| <= 1e-6 Eh)"

# DRAM traffic of one BF16x3 H_eff product (phase-1 + phase-2 kernels) from
# one ncu capture of a small case, scaled to the workload by its operator
# bytes; valid only while the kernel source is the one that was measured.
TRAFFIC = {
    # profiles/tc_gemm_bf16x3_l30_d1024.md: mean of nine products at cuts 14 and 15
    "l30_d1024": {"tc_cu": "5efed184da78b643", "form": "two_phase", "bytes_per_product": 21.47e9,
                  "source": "profiles/tc_gemm_bf16x3_l30_d1024.md (ncu, full-size workload, one-pass metrics)"},
}


def workload_name(W):
    return f"L={W['L']} N={W['N']} 2Sz={W['tsz']} D={W['D']} two-site steps around the mid-chain cut {W['b']}"


def src_hash(rel):
    import hashlib
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampler running during the timed region."""

    def __init__(self, index=0):
        self.rows = []
        self.proc = None
        self.index = index

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": len(self.rows)}
        try:
            sm = sorted(float(r[1]) for r in self.rows)
            out["sm_mhz"] = sm[len(sm) // 2]
            out["sm_max_mhz"] = max(float(r[2]) for r in self.rows)
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            reasons = set()
            for r in self.rows:
                for i, nme in enumerate(names):
                    if r[5 + i].lower() == "active":
                        reasons.add(nme)
            out["reasons"] = sorted(reasons)
        except Exception:
            pass
        return out


def sweep_compare(spec):
    """Full sweeps from one seeded MPS in FP64 and in the mixed form (sweep wall time, |dE|)."""
    import inputs
    import paper_2412_04676_gb300 as g
    L, N, D, nsw = (int(x) for x in spec.split(","))
    h, eri = inputs.make_integrals(L, 1000 + L)
    sites, dims = inputs.make_mps(L, N, 0, D, 77)
    out = {"workload": f"L={L} N={N} 2Sz=0 D={D}, {nsw} sweeps from the same random MPS"}
    for name, prec in (("fp64", g.FP64), ("mixed", g.MIXED_BF16X3)):
        ctx = g.Context(L, N, 0, D=D, precision=prec, offload=True, dav_tol=1e-8)
        ctx.load_integrals(h, eri)
        ctx.import_mps(sites, [1] * L)
        st = ctx.sweep(nsw, D)
        out[name] = {"ms_per_sweep": [s["ms_total"] for s in st], "energy": st[-1]["energy_last"],
                     "matvecs": sum(s["matvecs"] for s in st),
                     "ms_io_exposed": sum(s["ms_io_exposed"] for s in st),
                     "bytes_packed": sum(s["bytes_packed"] for s in st)}
        ctx.close()
    out["abs_dE"] = abs(out["mixed"]["energy"] - out["fp64"]["energy"])
    out["speedup_last_sweep"] = out["fp64"]["ms_per_sweep"][-1] / out["mixed"]["ms_per_sweep"][-1]
    # the environment-store options on the mixed form: recomputation from every
    # second environment, and a pinned store bounded to a quarter of one
    # sweep's saved bytes (the rest spilled to a file)
    bound = int(out["mixed"]["bytes_packed"] / nsw / 4)
    for name, kw in (("mixed_recompute2", dict(env_recompute=2)), ("mixed_spill", dict(host_store_bytes=bound))):
        ctx = g.Context(L, N, 0, D=D, precision=g.MIXED_BF16X3, offload=True, dav_tol=1e-8, **kw)
        ctx.load_integrals(h, eri)
        ctx.import_mps(sites, [1] * L)
        st = ctx.sweep(nsw, D)
        t = ctx.timers()
        out[name] = {"ms_per_sweep": [x["ms_total"] for x in st], "energy": st[-1]["energy_last"],
                     "ms_io_exposed": sum(x["ms_io_exposed"] for x in st),
                     "bytes_packed": sum(x["bytes_packed"] for x in st),
                     "recomputed": t["recompute_n"], "recompute_ms": t["recompute_ms"],
                     "spill_gb": t["spill_gbytes"], "restore_gb": t["restore_gbytes"],
                     "spill_wait_ms": t["spill_wait_ms"], "host_store_bytes": kw.get("host_store_bytes", 0)}
        out[name]["abs_dE_vs_mixed"] = abs(out[name]["energy"] - out["mixed"]["energy"])
        ctx.close()
    return out


# ---------------------------------------------------------------- oracle leg
def oracle_sample(seconds=20.0, max_steps=None, warmup=0):
    """The oracle's H_eff psi at L=10, N=10, D=256 (mid-chain cut 4), timed on host cores.

    Returns (useful TFLOP/s, cores, description, per-product seconds).
    """
    import numpy as np

    import inputs
    from oracle import dmrg as R
    from oracle import hamiltonian as H
    from oracle import mpo as M

    W = WORKLOADS["l10_d256"]
    L, N, tsz, D, b, seed = W["L"], W["N"], W["tsz"], W["D"], W["b"], W["seed"]
    h, eri = inputs.make_integrals(L, seed)
    mp = M.MPO(L, H.hamiltonian_terms(h, eri))
    sites, dims = inputs.make_mps(L, N, tsz, D, seed + 1, n_left=b)
    EL = R.build_left_envs(sites, dims, mp, b)[b]
    ER = R.build_right_envs(sites, dims, mp, b + 2, (N, tsz))[b + 2]
    He = R.Heff(EL, ER, dims, mp, b)
    flops = 0.0
    for (Q, Q2), bl, br in He.pairs:
        T, m1, m2 = bl.shape
        n2 = He.shape[Q2][1]
        n1 = He.shape[Q][1]
        flops += 2.0 * T * m1 * m2 * n2 + 2.0 * T * m1 * n2 * n1
    x = np.random.default_rng(0).normal(size=He.dim)
    for _ in range(warmup):
        He.matvec(x)
    times = []
    t0 = time.perf_counter()
    while True:
        t = time.perf_counter()
        He.matvec(x)
        times.append(time.perf_counter() - t)
        if max_steps is not None and len(times) >= max_steps:
            break
        if max_steps is None and time.perf_counter() - t0 >= seconds:
            break
    cores = os.cpu_count() or 0
    try:
        from threadpoolctl import threadpool_info
        cores = max(int(x.get("num_threads", 0)) for x in threadpool_info()) or cores
    except Exception:
        pass
    desc = (f"oracle H_eff psi products at L=10 N=10 2Sz=0 D=256 (mid-chain cut 4), dim {He.dim}, "
            f"{len(times)} products in {sum(times):.1f} s")
    return flops * len(times) / sum(times) / 1e12, cores, desc, times


def _oracle_child(q, seconds):
    try:
        q.put(oracle_sample(seconds))
    except Exception as e:  # reported, never fatal for the GPU arm
        q.put(("error", repr(e)))


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The oracle timed on the host cores: H_eff psi products at L=10, D=256.

    The oracle cannot build the environments of the larger workloads in
    bounded time, so its line always names the L=10 workload it ran; with
    --workload l10_d256 both arms run the same workload (like for like).
    """
    if rank != 0:
        return 0
    value, cores, desc, times = oracle_sample(max_steps=args.steps, warmup=args.warmup)
    ms = 1000.0 * sum(times) / len(times)
    ran = WORKLOADS["l10_d256"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"L={ran['L']} N={ran['N']} 2Sz={ran['tsz']} D={ran['D']} H_eff psi products "
                                   f"at the mid-chain cut {ran['b']} (oracle, FP64, host cores)",
                       "same_config_as_gpu_arm": args.workload == "l10_d256",
                       "gpu_arm_workload": workload_name(WORKLOADS[args.workload]),
                       "step": "one oracle H_eff psi product", "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm
def job_times(ms_dev, e2e_ms, world, device):
    """Slowest replica's device and end-to-end times (max over ranks)."""
    import torch
    vals = torch.tensor([ms_dev, e2e_ms], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(vals, op=dist.ReduceOp.MAX)
    return float(vals[0]), float(vals[1])


def job_value(world, flops_per_rank, ms):
    """Whole-job useful TFLOP/s: flops of all replicas over the slowest time."""
    return world * flops_per_rank / (ms * 1e-3) / 1e12

def config3_probe(device, max_matvec):
    """L=54, N=54, D=2048 at its mid-chain position (cut 26): one mixed Davidson.

    Environments are renormalised on the GPU from the seeded random MPS
    (offloaded as they are built); the Davidson starts from a random vector
    and runs BF16x3 products with sliced anchors.  Reported: its products'
    useful TFLOP/s, the device memory model of the position, and one product
    of each form against FP64 on the Davidson vector (relative residual and
    Rayleigh quotients).  Whole sweeps at this size need more device memory
    than one GB300 holds once the truncation concentrates the kept states
    (see the design notes), so the comparison is made at this position.
    """
    import torch

    import inputs
    import paper_2412_04676_gb300 as g
    W = WORKLOADS["l54_d2048"]
    L, N, tsz, D, b = W["L"], W["N"], W["tsz"], W["D"], W["b"]
    t0 = time.perf_counter()
    h, eri = inputs.make_integrals(L, W["seed"])
    sites, dims = inputs.make_mps(L, N, tsz, D, W["seed"] + 1, n_left=b)
    c = g.Context(L, N, tsz, D=D, precision=g.MIXED_BF16X3, offload=True, device=int(str(device).split(":")[-1]),
                  dav_tol=1e-6, dav_max_matvec=max_matvec)
    c.load_integrals(h, eri)
    c.import_mps(sites, [0] * b + [1] * (L - b))
    c.build_envs(b)
    t_env = time.perf_counter() - t0
    secs, info = c.tables(b)
    tm0 = c.timers()
    e, _, st, rc = c.davidson(b)
    tm1 = c.timers()
    psi, _ = c.get_psi()
    x = torch.from_numpy(psi).to(device)
    x = x / torch.linalg.norm(x)
    ym = c.apply_heff(b, x, precision=g.MIXED_BF16X3)
    ys = c.apply_heff(b, x, precision=g.SLICED_BF16)
    y64 = c.apply_heff(b, x, precision=g.FP64)
    tm2 = c.timers()
    n64 = float(torch.linalg.norm(y64))
    e64 = float(x @ y64)
    ms_bf = tm1["products_bf16x3_ms"] - tm0["products_bf16x3_ms"]
    n_bf = tm1["products_bf16x3_n"] - tm0["products_bf16x3_n"]
    out = {"workload": workload_name(W) + " (the mid-chain position only)",
           "environments_s": t_env, "psi_dim": info["dim"], "n_terms": info["n_terms"],
           "useful_gflop_per_product": info["useful_flops"] / 1e9,
           "device_memory_model_gb": {k: info[k] / 1e9 for k in ("mem_operators", "mem_planes_bf16x3",
                                                                 "mem_planes_sliced", "mem_x_fp64", "mem_x_tensor")},
           "davidson": {"energy": e, "status": rc, "matvecs": st["matvecs"], "resid": st["resid"],
                        "anchor_resid": st["anchor_resid"][:st["anchors"]], "ms_products": st["ms_matvec"]},
           "bf16x3_products": int(n_bf), "bf16x3_ms_per_product": ms_bf / max(n_bf, 1),
           "bf16x3_useful_tflops": info["useful_flops"] * n_bf / (ms_bf * 1e-3) / 1e12 if ms_bf else None,
           "sliced_ms_per_product": (tm1["products_sliced_ms"] - tm0["products_sliced_ms"])
                                    / max(tm1["products_sliced_n"] - tm0["products_sliced_n"], 1),
           "fp64_ms_per_product": tm2["products_fp64_ms"] - tm1["products_fp64_ms"],
           "vs_fp64": {"rel_resid_bf16x3": float(torch.linalg.norm(ym - y64)) / n64,
                       "rel_resid_sliced": float(torch.linalg.norm(ys - y64)) / n64,
                       "rayleigh_fp64": e64, "abs_dE_bf16x3": abs(float(x @ ym) - e64),
                       "abs_dE_sliced": abs(float(x @ ys) - e64)},
           "autotune": c.tune_info()}
    c.close()
    return out


def host_link_peak(device, nbytes=1 << 30, reps=5):
    """Pinned host <-> device copy bandwidth (plain cudaMemcpyAsync through torch), best of reps."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=device)
    out = {}
    for name, (dst, src) in (("d2h_gbs", (h, d)), ("h2d_gbs", (d, h))):
        best = 0.0
        for _ in range(reps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            dst.copy_(src, non_blocking=True)
            b.record()
            b.synchronize()
            best = max(best, nbytes / (a.elapsed_time(b) * 1e-3) / 1e9)
        out[name] = best
    out["bytes"] = nbytes
    out["how"] = "pinned host <-> device cudaMemcpyAsync of 1 GiB, best of 5"
    return out


def run_ours(args, rank, world, local_rank):
    import multiprocessing as mp_

    import numpy as np
    import torch

    import inputs
    import paper_2412_04676_gb300 as g
    from paper_2412_04676_gb300 import build

    cpu_q = None
    cpu_proc = None
    torch.cuda.set_device(local_rank)
    build.build()
    W = WORKLOADS[args.workload]
    L, N, tsz, D, b = W["L"], W["N"], W["tsz"], W["D"], W["b"]
    prec = g.MIXED_BF16X3 if args.precision == "mixed" else g.FP64
    h, eri = inputs.make_integrals(L, W["seed"])
    sites, dims = inputs.make_mps(L, N, tsz, D, W["seed"] + 1 + rank, n_left=b)

    def make_ctx():
        c = g.Context(L, N, tsz, D=D, precision=prec, offload=not args.no_offload, device=local_rank,
                      dav_tol=args.tol, dav_max_matvec=args.max_matvec, bf16x3_fused=args.fused)
        c.load_integrals(h, eri)
        c.import_mps(sites, [0] * b + [1] * (L - b))
        c.build_envs(b)
        return c

    ctx = make_ctx()
    secs, info = ctx.tables(b)
    pos = [b]
    dirs = [1]

    def one_step(c=None):
        c = c or ctx
        p, d = pos[0], dirs[0]
        st = c.step(p, d, D)
        pos[0] = p + d
        dirs[0] = -d
        return st

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        one_step()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local_rank)
    clocks.start()
    l0 = g.launch_count()
    tm0 = ctx.timers()
    stats = []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        stats.append(one_step())
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    l1 = g.launch_count()
    tm1 = ctx.timers()
    clk = clocks.stop()
    barrier()
    flops = sum(s["useful_flops"] for s in stats)
    ms_dev = sum(s["ms_device"] for s in stats)
    ms_mv = sum(s["ms_matvec"] for s in stats)
    nmv = sum(s["matvecs"] for s in stats)
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak_src = "of measured"
    except Exception:
        peaks = {}
        peak_src = "of fallback"
    hbm = peaks.get("hbm_gbs", 6800.0)
    bf16_burst = peaks.get("bf16_tflops", 1900.0)
    bf16_sust = peaks.get("bf16_tflops_sustained", 1700.0)
    # host link (NVLink-C2C) peak for the offload fraction
    link = None
    try:
        link = host_link_peak(f"cuda:{local_rank}")
    except Exception as e:  # measurement extra; never fatal
        link = {"error": repr(e)}
    # pack kernel throughput: HBM -> HBM on the environment the last step
    # produced, and the offload saves of the timed steps (pinned host memory)
    pack = None
    try:
        side, cut = (0, pos[0]) if dirs[0] == -1 else (1, pos[0] + 2)
        nbytes = ctx.pack_size(side, cut)
        io = ctx.io_stats()
        pk = {"offload_bytes": io["bytes_d2h"], "offload_ms": io["ms_save"],
              "offload_gbs": io["bytes_d2h"] / (io["ms_save"] * 1e-3) / 1e9 if io["ms_save"] > 0 else None}
        if pk["offload_gbs"] and link and link.get("d2h_gbs"):
            pk["offload_roofline"] = {"bound": "host link", "achieved": pk["offload_gbs"], "peak": link["d2h_gbs"],
                                      "unit": "GB/s", "frac": pk["offload_gbs"] / link["d2h_gbs"],
                                      "peak_source": "measured here: " + link["how"]}
        if nbytes > 0:
            dev = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            ctx.pack_env(side, cut, dev)
            t0 = ctx.io_stats()["ms_pack"]
            reps = 3
            for _ in range(reps):
                ctx.pack_env(side, cut, dev)
            ms = (ctx.io_stats()["ms_pack"] - t0) / reps
            gbs = 2 * nbytes / (ms * 1e-3) / 1e9
            pk.update({"bytes": nbytes, "hbm_ms": ms,
                       "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                                    "peak_source": f"{peak_src}: HBM copy bandwidth",
                                    "note": "read + write bytes of one packed environment, device to device"}})
        pack = pk
    except Exception as e:  # measurement extra; never fatal
        pack = {"error": repr(e)}
    # the mixed form against FP64 at the position the timed steps reached:
    # the relative residual of one product (BF16x3 and sliced against FP64 on
    # the current two-site vector) and the Rayleigh quotients; whole FP64
    # sweeps at the large workloads take hours on GB300's FP64 pipe
    fp64cmp = None
    if args.compare_fp64 and prec == g.MIXED_BF16X3:
        try:
            psi_c, pb_c = ctx.get_psi()
            xg = torch.from_numpy(psi_c).to(f"cuda:{local_rank}")
            xg = xg / torch.linalg.norm(xg)
            tq0 = ctx.timers()
            ym = ctx.apply_heff(pb_c, xg, precision=g.MIXED_BF16X3)
            ys = ctx.apply_heff(pb_c, xg, precision=g.SLICED_BF16)
            y64 = ctx.apply_heff(pb_c, xg, precision=g.FP64)
            ypb = ctx.apply_heff(pb_c, xg, precision=g.FP64_PER_BLOCK)
            tq1 = ctx.timers()
            # the two BF16x3 kernel forms on the same vector (comparison
            # forms, whichever the context runs), three products each after
            # one that builds the plan
            forms_ms = {}
            for name, code, key in (("two_phase", g.BF16X3_TWO_PHASE, "products_bf16x3_two_phase"),
                                    ("fused", g.BF16X3_FUSED, "products_bf16x3_fused")):
                ctx.apply_heff(pb_c, xg, precision=code)
                ta = ctx.timers()
                for _ in range(3):
                    yk = ctx.apply_heff(pb_c, xg, precision=code)
                tb = ctx.timers()
                forms_ms[name] = {"ms_per_product": (tb[key + "_ms"] - ta[key + "_ms"]) / 3,
                                  "rel_resid": float(torch.linalg.norm(yk - y64)) / float(torch.linalg.norm(y64))}
            n64 = float(torch.linalg.norm(y64))
            e64, em, es = float(xg @ y64), float(xg @ ym), float(xg @ ys)
            fp64cmp = {"position": pb_c, "rel_resid_bf16x3": float(torch.linalg.norm(ym - y64)) / n64,
                       "rel_resid_sliced": float(torch.linalg.norm(ys - y64)) / n64,
                       "rayleigh_fp64": e64, "abs_dE_bf16x3": abs(em - e64), "abs_dE_sliced": abs(es - e64),
                       "ms_fp64_product": tq1["products_fp64_ms"] - tq0["products_fp64_ms"],
                       "ms_fp64_per_block_product": tq1["products_fp64_per_block_ms"]
                                                    - tq0["products_fp64_per_block_ms"],
                       "per_block_bitwise_equal": bool(torch.equal(ypb, y64)),
                       "bf16x3_kernel_forms": dict(forms_ms, context_form="fused" if args.fused else "two_phase"),
                       "note": "one product of each form on the current two-site vector; the mixed Davidson's "
                               "energy comes from sliced anchor products (abs_dE_sliced)"}
        except Exception as e:  # measurement extra; never fatal
            fp64cmp = {"error": repr(e)}
    # end to end, on a fresh context from the same start (same warm-up, same
    # K steps, so the Davidson sees the same convergence progression): the
    # two-site vector is uploaded from pinned host memory and read back every
    # step through the public API
    ctx_tune = ctx.tune_info()
    ctx.close()
    ctx_e = make_ctx()
    pos[0], dirs[0] = b, 1
    for _ in range(args.warmup):
        one_step(ctx_e)
    psi, pb = ctx_e.get_psi()
    host = torch.from_numpy(psi).pin_memory()
    e2e_ms = 0.0
    e2e_flops = 0.0
    h2d = d2h = 0
    e2e_stats = []
    torch.cuda.synchronize()
    for _ in range(args.steps):
        t = time.perf_counter()
        ctx_e.set_psi(pos[0], host.numpy())
        st = one_step(ctx_e)
        e2e_stats.append(st)
        out, pb = ctx_e.get_psi()
        host = torch.from_numpy(out).pin_memory()
        e2e_ms += 1000.0 * (time.perf_counter() - t)
        e2e_flops += st["useful_flops"]
        h2d += psi.nbytes
        d2h += out.nbytes + 8
        psi = out
    ctx_e.close()
    sweep = None
    if args.sweep_config.strip("'\" ") and rank == 0:
        sweep = sweep_compare(args.sweep_config)
    cfg3 = None
    if args.config3 and rank == 0 and args.workload != "l54_d2048":
        try:
            cfg3 = config3_probe(f"cuda:{local_rank}", args.config3_max_matvec)
        except Exception as e:  # measurement extra; never fatal
            cfg3 = {"error": repr(e)}
    # the oracle runs only after the GPU measurements, so it never competes for host cores
    if rank == 0 and not args.no_cpu_baseline:
        ctx_mp = mp_.get_context("spawn")
        cpu_q = ctx_mp.Queue()
        cpu_proc = ctx_mp.Process(target=_oracle_child, args=(cpu_q, args.cpu_seconds), daemon=True)
        cpu_proc.start()
    ms_dev_max, e2e_max = job_times(ms_dev, e2e_ms, world, "cuda")
    value = job_value(world, flops, ms_dev_max)
    e2e_value = job_value(world, e2e_flops, e2e_max)
    if rank != 0:
        return 0
    flops_mv = info["useful_flops"]
    dt = {k: tm1[k] - tm0[k] for k in tm1}
    for k in ("tc_issued_gflop_p1", "tc_issued_gflop_p2", "tc_sliced_issued_gflop"):
        dt[k] = tm1[k]  # per product of the last prepared position, not accumulated
    # H_eff products of the timed steps by form (device time from the library)
    forms = {}
    for key in ("fp64", "bf16x3", "sliced"):
        n, ms, gf = dt[f"products_{key}_n"], dt[f"products_{key}_ms"], dt[f"products_{key}_gflop"]
        if n > 0 and ms > 0:
            forms[key] = {"products": int(round(n)), "ms": ms, "useful_gflop": gf,
                          "useful_tflops": gf / ms}
    roofs = {}
    if "fp64" in forms:
        a = forms["fp64"]["useful_tflops"]
        roofs["fp64"] = {"bound": "alu", "achieved": a, "peak": args.fp64_peak, "unit": "TFLOP/s",
                         "frac": a / args.fp64_peak, "traffic": None, "ms": forms["fp64"]["ms"],
                         "kernel": "gemm_f64_kernel: FP64 H_eff product (phase-1 + phase-2 launches)",
                         "peak_source": "of measured: cuBLAS DGEMM 8192^3 on a GB300"}
    if "bf16x3" in forms:
        f = forms["bf16x3"]
        a, n = f["useful_tflops"], f["products"]
        gb, xgb = dt["products_bf16x3_gbytes"], dt["products_bf16x3_x_gbytes"]
        peak = bf16_sust / 3.0
        tr = TRAFFIC.get(args.workload)
        traffic = None
        if (tr and tr.get("tc_cu") == src_hash("paper_2412_04676_gb300/csrc/tc.cu")
                and tr.get("form") == ("fused" if args.fused else "two_phase")):
            traffic = tr["bytes_per_product"]
        roofs["bf16x3"] = {
            "bound": "tensor", "achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
            "traffic": traffic, "traffic_source": tr["source"] if traffic else "no capture of this kernel build",
            "ms": f["ms"], "launches": n,
            "kernel": ("tc_fused_kernel (+ split, reduce): BF16x3 H_eff product, X kept in TMEM" if args.fused else
                       "tc_gemm_kernel<0, 1> + <0, 2> (+ split, reduce): BF16x3 H_eff product in two kernels"),
            "peak_source": f"{peak_src}: bf16 sustained / 3 (three split products per useful flop; "
                           "the product is timed inside whole steps)",
            "algorithmic_bytes_per_product": gb / n * 1e9,
            "bytes_note": "operators read once as BF16 hi+lo (4 B/element), psi in and H psi out (FP64)",
            "hbm_view": {"achieved": gb / (f["ms"] * 1e-3), "peak": hbm, "unit": "GB/s",
                         "frac": gb / (f["ms"] * 1e-3) / hbm, "peak_source": f"{peak_src}: HBM copy bandwidth"},
            "traffic_view": ({"achieved": traffic / (f["ms"] / n * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                              "frac": traffic / (f["ms"] / n * 1e-3) / 1e9 / hbm,
                              "peak_source": f"{peak_src}: HBM copy bandwidth",
                              "note": "measured DRAM bytes per product (traffic) over its device time in the timed "
                                      "steps: how close the kernel runs to HBM given the bytes it moves"}
                             if traffic else None),
            "x_overhead_bytes_per_product": xgb / n * 1e9,
            "x_overhead_note": "two-kernel form: phase-1 intermediate X written and read once (BF16 hi+lo), "
                               "not algorithmic; 0 for the fused kernel",
            "intensity_flop_per_byte": 3.0 * f["useful_gflop"] / gb if gb else None,
            "ridge_flop_per_byte": bf16_sust * 1e3 / hbm,
            "issued_tflops": (dt["tc_issued_gflop_p1"] + dt["tc_issued_gflop_p2"]) * n / f["ms"],
            "issued_note": "bf16 MMA flops of whole 128-row tiles at the MMA width, padding included"}
    if "sliced" in forms:
        a = forms["sliced"]["useful_tflops"]
        roofs["sliced"] = {"bound": "tensor", "achieved": a, "peak": bf16_sust / 10.0, "unit": "TFLOP/s",
                           "frac": a / (bf16_sust / 10.0), "traffic": None, "ms": forms["sliced"]["ms"],
                           "kernel": "tc_gemm_kernel<1>: sliced H_eff product, Davidson anchors",
                           "peak_source": f"{peak_src}: bf16 sustained / 10 (ten slice products per useful flop)",
                           "issued_tflops": dt["tc_sliced_issued_gflop"] * forms["sliced"]["products"]
                                            / forms["sliced"]["ms"]}
    env_ms = dt["enlarge_dev"] + dt["renorm_dev"]
    if env_ms > 0:
        gf64 = dt["enlarge_gflop"] + dt["renorm_gflop"]
        gftc = dt["renorm_tc_gflop"] + dt["enlarge_tc_gflop"]
        a = (gf64 + gftc) / env_ms
        roofs["environments"] = {"bound": "alu" if gftc == 0 else "alu+tensor", "achieved": a,
                                 "peak": args.fp64_peak if gftc == 0 else None, "unit": "TFLOP/s",
                                 "frac": a / args.fp64_peak if gftc == 0 else None, "traffic": None, "ms": env_ms,
                                 "fp64_gflop": gf64, "tensor_gflop": gftc,
                                 "kernel": "gemm_f64_kernel + copy_sum_kernel (+ tc_gemm_kernel<1, 3> for the "
                                           "sliced share): enlargement and renormalisation",
                                 "peak_source": "of measured: cuBLAS DGEMM 8192^3 on a GB300 (FP64 share)"}
    # the dominant kernel by device time in the timed steps
    roof = max(roofs.values(), key=lambda r: r["ms"]) if roofs else None
    cpu = None
    if cpu_q is not None:
        try:
            r = cpu_q.get(timeout=args.cpu_seconds + 240)
            if r and r[0] != "error":
                cpu = {"value": r[0], "unit": "TFLOP/s", "cores": r[1], "kind": "oracle", "sample": r[2],
                       "same_config": args.workload == "l10_d256"}
            else:
                cpu = {"value": None, "unit": "TFLOP/s", "cores": 0, "kind": "oracle", "sample": str(r)}
        except Exception as e:
            cpu = {"value": None, "unit": "TFLOP/s", "cores": 0, "kind": "oracle", "sample": f"timeout {e!r}"}
    status = [s["dav_status"] for s in stats]
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_dev_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == g.FP64 else "bf16->f32",
        "data": "synthetic",
        "config": {"workload": workload_name(W),
                   "precision": args.precision, "offload": not args.no_offload,
                   "environments": "renormalised on the GPU from a seeded random isometric MPS with the "
                                   f"D={D} sector distribution",
                   "l2": "operands larger than L2 (enlarged operators > 1 GB)" if info["operator_bytes"] > 2e9
                         else "small workload: operands may fit in L2",
                   "parallelism": f"replicas x{world}", "psi_dim": info["dim"], "n_terms": info["n_terms"],
                   "useful_gflop_per_product_at_start": flops_mv / 1e9,
                   "device_memory_model_gb": {k: info[k] / 1e9 for k in ("mem_operators", "mem_planes_bf16x3",
                                                                          "mem_planes_sliced", "mem_x_fp64",
                                                                          "mem_x_tensor")}},
        "e2e": {"value": e2e_value, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d // args.steps,
                "d2h_bytes_per_step": d2h // args.steps},
        "gpu_launches": int(l1 - l0),
        "roofline": roof,
        "roofline_all": roofs,
        "cpu_baseline": cpu,
        "clocks": clk,
        "davidson": {"converged_steps": sum(1 for x in status if x == 0), "steps": len(status),
                     "at_product_limit": sum(1 for x in status if x == 1),
                     "at_precision_floor": sum(1 for x in status if x == 2),
                     "status_note": "0: residual <= tol; 1: product limit; 2: mixed form stopped at its "
                                    "rounding floor (an anchor that did not cut the exact residual by a fifth, or six "
                                    "anchors) above tol",
                     "status_per_step": status, "matvecs_per_step": [s["matvecs"] for s in stats],
                     "resid_per_step": [s["resid"] for s in stats],
                     "anchor_resid_per_step": [s["anchor_resid"][:s["anchors"]] for s in stats],
                     "max_matvec": args.max_matvec,
                     "tol": args.tol},
        "host_link": link,
        "fp64_compare": fp64cmp,
        "autotune": ctx_tune,
        "pack": pack,
        "sweep": sweep,
        "config3": cfg3,
        "detail": {"matvec_tflops": flops / (ms_mv * 1e-3) / 1e12 if ms_mv else 0.0, "matvecs": nmv,
                   "ms_matvec": ms_mv, "ms_device": ms_dev,
                   "wall_s": t_wall, "energy": stats[-1]["energy"],
                   "ms_io_exposed": sum(s["ms_io_exposed"] for s in stats),
                   "bytes_packed_per_step": sum(s["bytes_packed"] for s in stats) / args.steps,
                   "ms_truncate": sum(s["ms_truncate"] for s in stats),
                   "ms_renorm": sum(s["ms_renorm"] for s in stats),
                   "timers_ms": dt, "products": forms,
                   "e2e_steps_matvecs": [s["matvecs"] for s in e2e_stats],
                   "e2e_steps_ms": [s["ms_device"] for s in e2e_stats]},
    }
    print(json.dumps(line), flush=True)
    if cpu_proc is not None:
        cpu_proc.join(timeout=5)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-offload", action="store_true")
    ap.add_argument("--fused", action="store_true",
                    help="BF16x3 products in one fused kernel with X kept in TMEM (default: two kernels, X in HBM)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-matvec", type=int, default=120)
    ap.add_argument("--fp64-peak", type=float, default=1.0975)
    ap.add_argument("--no-config3", dest="config3", action="store_false",
                    help="skip the L=54, D=2048 mid-chain Davidson and its FP64 comparison")
    ap.add_argument("--config3-max-matvec", type=int, default=200,
                    help="product limit of the L=54, D=2048 Davidson (it starts from a random vector)")
    ap.add_argument("--no-compare-fp64", dest="compare_fp64", action="store_false",
                    help="skip the sampled mixed-vs-FP64 product comparison")
    ap.add_argument("--sweep-config", default="14,14,384,4",
                    help="L,N,D,sweeps of the FP64-vs-mixed sweep comparison ('' to skip)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
    else:
        rc = run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
