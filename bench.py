"""Benchmark: Gcell-updates/s of block-relaxation sweeps on a 256^3 grid (one GB300 per rank).

Headline workload: 256^3 interior cells, a = (1,1,1), x-line block Jacobi (omega = 0.8),
FP64 (the paper's precision), b = h^2 f and u0 from seeded U[-1,1] draws; one step = one
library call of 50 sweeps.  With N ranks (torchrun) every rank sweeps its own replica (no
data-path collective: the grids are independent), so `value` is N x cells x sweeps /
(max-over-ranks time).

Also reported on the same JSON line:
  roofline     -- the binding roof of the FP64 sweep kernel: FP64 pipe operations (7 per
                  cell: gather 4, elimination 1 each way, update 1) per launch / average
                  launch time, against the FP64 FMA rate measured in the same run;
  roofline_hbm -- the same kernel against the HBM roof (24 algorithmic bytes per cell);
  e2e          -- the same metric through the host-buffer C-ABI entry point, with the H2D
                  copies of u and b and the D2H copy of u inside the timed region;
  cpu_baseline -- the FP64 CPU oracle on the host cores on a bounded slab of the grid;
  clocks       -- nvidia-smi samples taken during the timed region;
  variants     -- other method / dtype / coefficient / block combinations, each with its
                  error against the FP64 oracle and, where timed, the oracle's own rate.

`--impl reference` times the FP64 CPU oracle instead (rank 0 only), on the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

METRIC = "Gcell-updates/s per sweep & % HBM roofline; FP64 vs mixed at equal residual"
UNIT = "Gcell-updates/s"
N = 256
SWEEPS_PER_STEP = 50
COEFFS = (1.0, 1.0, 1.0)
L2_BYTES = 129e6


def _peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _bf16_peak():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return float(json.loads(p.read_text())["bf16_tflops"])
    return 1900.0


def _live_copy_gbs():
    """Device-to-device copy bandwidth on this machine right now (read + write bytes, best of 10)."""
    import torch

    n = 1 << 28  # 1 GiB of float32
    a = torch.empty(n, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    b.copy_(a)
    best = 1e30
    for _ in range(10):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.copy_(a)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    return 2 * 4 * n / (best / 1e3) / 1e9


def max_over_ranks(x: float, ws: int, device="cuda") -> float:
    """Largest value of x over all ranks (identity when running alone)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells_per_rank: int, sweeps: int, slowest_s: float, ws: int) -> float:
    """Gcell-updates/s of the whole job: every rank sweeps its own replica, the job ends with
    the slowest rank."""
    return ws * cells_per_rank * sweeps / slowest_s / 1e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples (SM clock, throttle reasons) while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _inputs(dtype_str):
    """Seeded synthetic u0 and b = h^2 f of the 256^3 workload, on the current CUDA device."""
    import torch

    from brs_inputs import initial_guess, rhs

    td = torch.float64 if dtype_str == "f64" else torch.float32
    u0 = torch.from_numpy(initial_guess((N, N, N))).to(td)
    b = torch.from_numpy(rhs((N, N, N))).to(td)
    return u0, b


def _time_sweeps(ctx, u, b, steps, warmup, sweeps, stream, barrier=None):
    import torch

    for _ in range(warmup):
        ctx.sweep(u, b, sweeps, stream=stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.sweep(u, b, sweeps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    return e0.elapsed_time(e1)  # ms


def _cpu_baseline(budget_s: float = 10.0):
    """FP64 oracle x-line Jacobi on a 256 x 256 x 8 slab of the workload (bounded sample)."""
    import oracle
    from brs_inputs import initial_guess, rhs

    oracle.build()
    nz = 8
    u = initial_guess((N, N, N))[:nz].copy()
    b = rhs((N, N, N))[:nz].copy()
    oracle.sweep(u, b, COEFFS, block="line", method="jacobi", omega=0.8)  # warm
    t0 = time.perf_counter()
    sweeps = 0
    while True:
        u = oracle.sweep(u, b, COEFFS, block="line", method="jacobi", omega=0.8)
        sweeps += 1
        if time.perf_counter() - t0 >= budget_s or sweeps >= 100000:
            break
    dt = time.perf_counter() - t0
    cells = N * N * nz
    return {"value": cells * sweeps / dt / 1e9, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"FP64 oracle x-line block Jacobi, {sweeps} sweeps of a 256x256x{nz} slab "
                      f"(same cells/line and coefficients as the 256^3 workload), {dt:.1f} s"}


# ---------------------------------------------------------------------------------------
# CPU-baseline legs: the FP64 oracle timed beside each workload variant on a bounded sample,
# and the error of the variant's GPU result against it.  Block Jacobi and the deterministic
# two-colour Gauss-Seidel orders are compared element by element on sampled blocks (the
# oracle sweeps a sub-grid of the blocks around each one; a block's value after one sweep
# depends only on blocks within distance 1 (Jacobi) or 2 (two colours), so cut sub-grid
# edges never reach the sampled block).  Chaotic Gauss-Seidel, which no sequential order
# reproduces, is placed in its residual bracket on a small grid: between the ordered
# Gauss-Seidel sweeps and Jacobi with omega = 1.

def _orc():
    import oracle

    oracle.build()
    return oracle


def _block_dims(blk, box, shape):
    nz, ny, nx = shape
    return {"line": (nx, 1, 1), "plane": (nx, ny, 1), "yline": (1, ny, 1),
            "zline": (1, 1, nz)}.get(blk, tuple(int(v) for v in box))


def _orc_sweep(orc, u, b, a, blk, box, method, omega):
    if blk in ("line", "plane"):
        return orc.sweep(u, b, a, block=blk, method=method, omega=omega)
    return orc.sweep(u, b, a, block="box", method=method, omega=omega,
                     box=_block_dims(blk, box, u.shape))


def _rel_err(got, ref):
    import numpy as np

    s = float(np.max(np.abs(ref)))
    return float(np.max(np.abs(got - ref))) / (s if s > 0 else 1.0)


def _sampled_block_err(orc, blk, box, a, method, omega, u, b, got, picks, nsweeps=1):
    """Largest error of `got` (the GPU's iterate after nsweeps sweeps from u) over the sampled
    blocks `picks` (block indices (bi, bj, bk)), relative to the oracle block's max-norm and
    relative to the input's max-norm; oracle cells and seconds.  A block after s sweeps
    depends only on blocks within s of it (2 s in the zebra order)."""
    import numpy as np

    nz, ny, nx = u.shape
    bx, by, bz = _block_dims(blk, box, u.shape)
    nb = (nx // bx, ny // by, nz // bz)
    zebra = method == "gs_zebra"
    rad = (2 if zebra else 1) * nsweeps
    worst, worst_in, cells, secs = 0.0, 0.0, 0, 0.0
    scale_in = float(np.max(np.abs(u)))
    for pk in picks:
        lo = [max(0, c - rad) for c in pk]
        hi = [min(n, c + rad + 1) for n, c in zip(nb, pk)]
        if zebra and sum(lo) % 2:  # keep the sub-grid's colours those of the grid
            d = next(q for q in range(3) if lo[q] > 0)
            lo[d] -= 1
        sl = (slice(lo[2] * bz, hi[2] * bz), slice(lo[1] * by, hi[1] * by),
              slice(lo[0] * bx, hi[0] * bx))
        t0 = time.perf_counter()
        ref = np.ascontiguousarray(u[sl])
        bs = np.ascontiguousarray(b[sl])
        for _ in range(nsweeps):
            ref = _orc_sweep(orc, ref, bs, a, blk, box, method, omega)
        secs += time.perf_counter() - t0
        cells += ref.size * nsweeps  # cell-updates
        c = [(pk[q] - lo[q]) for q in range(3)]
        own = (slice(c[2] * bz, (c[2] + 1) * bz), slice(c[1] * by, (c[1] + 1) * by),
               slice(c[0] * bx, (c[0] + 1) * bx))
        g = got[pk[2] * bz:(pk[2] + 1) * bz, pk[1] * by:(pk[1] + 1) * by,
                pk[0] * bx:(pk[0] + 1) * bx]
        worst = max(worst, _rel_err(g, ref[own]))
        worst_in = max(worst_in, float(np.max(np.abs(g - ref[own]))) / scale_in)
    return worst, worst_in, cells, secs


def _picks(blk, box, shape, k=6):
    import numpy as np

    bx, by, bz = _block_dims(blk, box, shape)
    nb = (shape[2] // bx, shape[1] // by, shape[0] // bz)
    rng = np.random.default_rng(17)
    out = [(0, 0, 0), (nb[0] - 1, nb[1] - 1, nb[2] - 1)]
    out += [tuple(int(rng.integers(0, n)) for n in nb) for _ in range(k - 2)]
    return out


def _gpu_sweeps(brs, stream, blk, meth, dt, a, math, box, u_np, b_np, nsweeps=1):
    import torch

    td = torch.float64 if dt == "f64" else torch.float32
    nz, ny, nx = u_np.shape
    ut = torch.from_numpy(u_np).to(td).cuda()
    bt = torch.from_numpy(b_np).to(td).cuda()
    with brs.Context(nx, ny, nz, a, block=blk, method=meth, dtype=dt, plane_math=math,
                     box=box) as c:
        c.sweep(ut, bt, nsweeps, stream=stream)
        torch.cuda.synchronize()
        if c.last_error() != 0:
            raise RuntimeError("device status raised")
    return ut.double().cpu().numpy()


def _deterministic_gs(blk, dt):
    """Gauss-Seidel forms that visit the blocks in two colours (the oracle's zebra order):
    FP64 x-lines (red-black lines), xy-planes (even, then odd planes) and boxes."""
    return blk in ("plane", "box") or (blk == "line" and dt == "f64")


def _bracket_leg(orc, brs, stream, blk, dt, a, math, box, shape, sweeps=3):
    """Chaotic GS on a small grid: GPU residual after each sweep against the oracle's
    Jacobi (omega = 1) and ordered Gauss-Seidel residuals from the same start."""
    import numpy as np
    import torch

    from brs_inputs import initial_guess, rhs

    nz, ny, nx = shape
    u0 = initial_guess(shape)
    b = rhs(shape)
    if dt == "f32":
        u0, b = u0.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    ref = {}
    for m in ("jacobi", "gs_lex", "gs_zebra", "gs_reverse"):
        u, rs = u0, []
        for _ in range(sweeps):
            u = _orc_sweep(orc, u, b, a, blk, box, m, 1.0)
            rs.append(orc.residual_norm(u, b, a))
        ref[m] = np.array(rs)
    secs = time.perf_counter() - t0
    td = torch.float64 if dt == "f64" else torch.float32
    ut, bt = torch.from_numpy(u0).to(td).cuda(), torch.from_numpy(b).to(td).cuda()
    got = []
    with brs.Context(nx, ny, nz, a, block=blk, method="gs", dtype=dt, plane_math=math,
                     box=box) as c:
        for _ in range(sweeps):
            c.sweep(ut, bt, 1, stream=stream)
            got.append(orc.residual_norm(ut.double().cpu().numpy(), b, a))
    got = np.array(got)
    lo = np.minimum(np.minimum(ref["gs_lex"], ref["gs_zebra"]), ref["gs_reverse"])
    cells = 4 * sweeps * int(np.prod(shape))
    return ({"metric": "residual bracket of chaotic GS (not reproducible element by element)",
             "grid": list(shape), "sweeps": sweeps,
             "ratio_to_jacobi_omega1": (got / ref["jacobi"]).tolist(),
             "ratio_to_best_ordered_gs": (got / lo).tolist(),
             "within_bracket": bool(np.all(got <= 1.1 * ref["jacobi"])
                                    and np.all(got >= 0.9 * lo))},
            {"value": cells / secs / 1e9, "unit": UNIT, "cores": orc.num_threads(),
             "kind": "oracle",
             "sample": f"oracle Jacobi and three ordered GS sweeps x{sweeps} on a "
                       f"{nx}x{ny}x{nz} grid, {secs:.2f} s"})


def _grid_cpu_leg(brs, stream, blk, meth, dt, a, math, box, nsweeps=1):
    """cpu_baseline and err_vs_oracle of a 256^3 variant (nsweeps sweeps in one call)."""
    import numpy as np

    orc = _orc()
    if meth == "gs" and not _deterministic_gs(blk, dt):
        # large enough that the persistent kernel marches several planes per CTA, as at 256^3
        small = {"line": (128, 256, 256), "yline": (128, 256, 64), "zline": (256, 128, 64)}.get(
            blk, (128, 256, 256))
        return _bracket_leg(orc, brs, stream, blk, dt, a, math, box, small)
    u_np, b_np = (x.double().numpy() for x in _inputs(dt))
    got = _gpu_sweeps(brs, stream, blk, meth, dt, a, math, box, u_np, b_np, nsweeps)
    omet = "jacobi" if meth == "jacobi" else "gs_zebra"
    om = 0.8 if meth == "jacobi" else 1.0
    err, err_in, cells, secs = _sampled_block_err(orc, blk, box, a, omet, om, u_np, b_np, got,
                                                  _picks(blk, box, u_np.shape), nsweeps)
    tol = 1e-12 if dt == "f64" else ((2.0 ** -10 if nsweeps > 1 else 2.0 ** -11)
                                     if math == "tf32" else 1e-5)
    what = "one sweep" if nsweeps == 1 else f"{nsweeps} sweeps in one call"
    rec = {"metric": f"relative max-norm after {what}, sampled blocks vs the oracle's "
                     + ("zebra-order GS" if meth == "gs" else "Jacobi"),
           "value": err, "tolerance": tol, "blocks_sampled": 6}
    if meth == "gs":
        # omega = 1 leaves only the block solve, whose result is much smaller than the input
        # for rough data; rounding scales with the input, so report both normalisations
        rec["value_rel_to_input"] = err_in
        rec["tolerance_applies_to"] = "value_rel_to_input (GS acceptance is the bracket and " \
                                      "convergence; the 1e-12 / 1e-5 bars are Jacobi's)"
    return (rec,
            {"value": cells / secs / 1e9, "unit": UNIT, "cores": orc.num_threads(),
             "kind": "oracle",
             "sample": f"oracle {omet} sweeps ({nsweeps} each) of the sub-grids around 6 "
                       f"sampled blocks ({cells} cell-updates, {secs:.2f} s)"})


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from brs_inputs import initial_guess, rhs

    oracle.build()
    nz = 4  # bounded slab per step: 256 x 256 x 4 cells
    u = initial_guess((N, N, N))[:nz].copy()
    b = rhs((N, N, N))[:nz].copy()
    for _ in range(args.warmup):
        u = oracle.sweep(u, b, COEFFS, block="line", method="jacobi", omega=0.8)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u = oracle.sweep(u, b, COEFFS, block="line", method="jacobi", omega=0.8)
    dt = time.perf_counter() - t0
    cells = N * N * nz
    val = cells * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "grid256_iso: 256^3 x-line block Jacobi a=(1,1,1) omega=0.8; "
                                   "reference step = one FP64 oracle sweep of a 256x256x4 slab",
                       "nx": N, "ny": N, "nz": N},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": "one x-line Jacobi sweep of a 256x256x4 slab per step"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _traffic_record(profile: str, sources):
    """Per-launch DRAM bytes of a kernel from its committed ncu summary, if still current:
    the summary records a hash of the kernel's sources, and a changed kernel gives None."""
    import hashlib
    import re

    rec = ROOT / "profiles" / profile
    if not rec.exists():
        return None
    text = rec.read_text()
    m_b = re.search(r"^traffic_per_launch_bytes:\s*(\d+)", text, re.M)
    m_h = re.search(r"^source_sha256_16:\s*([0-9a-f]+)", text, re.M)
    h = hashlib.sha256()
    for src in sources:
        h.update((ROOT / "paper_1208_1975_gb300" / "csrc" / src).read_bytes())
    if not (m_b and m_h) or m_h.group(1) != h.hexdigest()[:16]:
        return None  # the kernel changed since the counters were taken
    return int(m_b.group(1))


def _live_fp64_fma_rate(brs, stream):
    """FP64 FMAs per second on this GPU right now: the library's FMA-bound probe kernel
    (8 independent chains per thread, every SM full), best of 5 CUDA-event timings."""
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks, iters = sms * 8, 2048
    out = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    h = _stream_int(stream)
    for _ in range(2):
        if brs.brsmooth_probe_fp64_fma(out.data_ptr(), blocks, iters, h) != 0:
            raise RuntimeError("FP64 FMA probe failed to launch")
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        brs.brsmooth_probe_fp64_fma(out.data_ptr(), blocks, iters, h)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return blocks * 256 * iters * 8 / (best / 1e3)


def _stream_int(stream):
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)


def _launch_ms(ctx, u, b, stream, k=50, reps=5):
    """Average duration of one sweep launch inside a call, as the timed steps run them
    (back-to-back dependent launches): (T(k+1 sweeps) - T(1 sweep)) / k per call, median
    of `reps`, CUDA events on the launching stream.  Both calls pay the same per-call
    copies, so the difference is k sweep launches."""
    import torch

    def one(ns):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.sweep(u, b, ns, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    one(1), one(k + 1)
    d = sorted(one(k + 1) - one(1) for _ in range(reps))
    return d[len(d) // 2] / k


def _rate(cells, sweeps, ms):
    return cells * sweeps / (ms / 1e3) / 1e9


_FMA = {}


def _fma_rate(brs, stream):
    """FP64 FMAs per second, measured once per run by the probe kernel."""
    if "rate" not in _FMA:
        _FMA["rate"] = _live_fp64_fma_rate(brs, stream)
    return _FMA["rate"]


def _plane_form(ny):
    """The plane solve the library runs: 1 = x sine transform + y tridiagonal solves (two
    dense n x n contractions per plane), 2 = 2D sine basis (four)."""
    return 1 if os.environ.get("BRSMOOTH_PLANE_FORM", "1") == "1" and ny <= 512 else 2


def _box_fma_per_cell(box, dt, math):
    """Multiply-adds per cell of the box product as the library runs it: n for the full
    product; sum over the 8 parity classes of n_c^2 / n on CUDA cores where that saves half
    the work and a class has 16+ cells (BRSMOOTH_BOX_FOLD=0: the full product)."""
    n = box[0] * box[1] * box[2]
    cuda_cores = dt == "f64" or math == "simt" or (math == "auto" and (n % 4 or n < 32))
    if not cuda_cores or os.environ.get("BRSMOOTH_BOX_FOLD", "1") == "0":
        return float(n)
    sizes = []
    for cl in range(8):
        nc = 1
        for d in range(3):
            h = box[d] // 2
            nc *= h if (cl >> d) & 1 else box[d] - h
        sizes.append(nc)
    work = sum(x * x for x in sizes)
    if 2 * work > n * n or max(sizes) < 16:
        return float(n)
    return work / n


def _plane_modes_min(dt, math):
    """Smallest sweep count per call for which the library runs the x-sine form (plane
    contexts whose y rows TMA can stage; 0 when switched off by BRSMOOTH_PLANE_MODES=0)."""
    if os.environ.get("BRSMOOTH_PLANE_MODES", "1") == "0":
        return 0
    if os.environ.get("BRSMOOTH_PLANE_MODES_MIN"):
        return max(1, int(os.environ["BRSMOOTH_PLANE_MODES_MIN"]))
    return 3 if dt == "f32" and math in ("auto", "tf32", "3xtf32") else 2


def _variant_grid(brs, stream, barrier, peak, blk, meth, dt, a, steps, sweeps, math="auto",
                  box=(0, 0, 0)):
    """One 256^3 workload variant: steps x sweeps sweeps timed with CUDA events.  For the
    x-sine form of plane calls, calls of fewer sweeps are timed too: the difference gives
    the time of one mode-line sweep and the fixed cost of a call's three transforms."""
    uv0, bv = _inputs(dt)
    uv, bv = uv0.cuda(), bv.cuda()
    mmin = _plane_modes_min(dt, math) if blk == "plane" else 0
    modes = mmin > 0 and sweeps >= mmin
    s_lo = max(mmin, sweeps // 5)
    es = 8 if dt == "f64" else 4
    with brs.Context(N, N, N, a, block=blk, method=meth, dtype=dt, plane_math=math,
                     box=box) as vc:
        vms = _time_sweeps(vc, uv, bv, steps, 1, sweeps, stream, barrier)
        if modes and s_lo < sweeps:
            lo_ms = _time_sweeps(vc, uv, bv, steps, 1, s_lo, stream, barrier)
            sweep_ms = (vms - lo_ms) / (steps * (sweeps - s_lo))
            fixed_ms = vms / steps - sweeps * sweep_ms
    rate = _rate(N ** 3, sweeps * steps, vms)
    out = {"workload": "grid256", "block": blk, "method": meth, "dtype": dt, "coeffs": a,
           "value": rate, "unit": UNIT, "hbm_frac": rate * 3 * es / peak,
           "sweeps_per_call": sweeps}
    fma = _fma_rate(brs, stream) / 1e9 if dt == "f64" else None
    if blk == "box":
        # the dense block product: n multiply-adds per cell, n = bx by bz (Alg. 2 step 2); on
        # CUDA cores by parity classes where the library uses them: sum_c n_c^2 / n
        nfull = box[0] * box[1] * box[2]
        nb = _box_fma_per_cell(box, dt, math)
        out["box"] = list(box)
        out["plane_math"] = math
        out["fma_per_cell"] = nb
        out["parity_classes"] = nb < nfull
        out["tflops"] = rate * 2 * nb / 1e3
        if math in ("tf32", "3xtf32"):
            passes = 3 if math == "3xtf32" else 1
            tf32_peak = _bf16_peak() / 2
            out["tensor_tflops"] = out["tflops"] * passes
            out["tensor_frac_of_tf32_peak"] = out["tensor_tflops"] / tf32_peak
            out["tf32_peak_tflops"] = tf32_peak
        if dt == "f64":
            out["alu_frac_of_fp64_fma_rate"] = rate * nb / fma
    if blk == "plane" and math == "auto":
        math = "3xtf32" if dt == "f32" and N % 32 == 0 else "simt"  # the library's choice
    if blk == "plane" and modes:
        # x-sine form: per call, the x-DST of b and of u and the inverse x-DST of u (nx
        # multiply-adds per cell each; FP64 splits each by the basis's even/odd symmetry into
        # two half-size products, (ceil(nx/2)^2 + floor(nx/2)^2) / nx per cell), then
        # mode-line sweeps: 3 words per cell, HBM-bound in FP32
        passes = 3 if math == "3xtf32" else 1
        fold = dt == "f64" and os.environ.get("BRSMOOTH_MODE_FOLD", "1") != "0"
        fma_t = ((N - N // 2) ** 2 + (N // 2) ** 2) / N if fold else float(N)
        out["plane_form"] = "x-sine basis: 3 transforms per call + mode-line sweeps"
        out["plane_math"] = math
        out["transform_fma_per_cell"] = fma_t
        out["tflops"] = 6.0 * fma_t * rate / sweeps / 1e3
        if s_lo < sweeps:
            out["mode_sweep_us"] = sweep_ms * 1e3
            out["mode_sweep_gcell"] = N ** 3 / (sweep_ms / 1e3) / 1e9
            out["mode_sweep_hbm_frac"] = 3 * es * N ** 3 / (sweep_ms / 1e3) / 1e9 / peak
            out["transforms_ms_per_call"] = fixed_ms
            out["transforms_timing"] = (f"calls of {sweeps} and {s_lo} sweeps, the difference "
                                        "per sweep and the remainder per call")
            if math in ("tf32", "3xtf32"):
                out["transforms_tensor_tflops"] = (3 * 2.0 * N * N ** 3 * passes
                                                   / (fixed_ms / 1e3) / 1e12)
            if dt == "f64":
                out["transforms_frac_of_fp64_fma_rate"] = (3.0 * fma_t * N ** 3
                                                           / (fixed_ms / 1e3) / (fma * 1e9))
    elif blk == "plane":
        # dense contractions per plane: form 1 (x sine transform + y tridiagonal solves) runs
        # the forward and inverse x transforms, nx multiply-adds per cell each; form 2 (2D
        # sine basis) runs four, 2 (nx + ny) multiply-adds per cell in all
        form = _plane_form(N)
        flops_per_cell = 4.0 * N if form == 1 else 4.0 * (N + N)
        out["plane_form"] = form
        out["plane_math"] = math
        out["tflops"] = flops_per_cell * rate / 1e3
        if math in ("tf32", "3xtf32"):
            # tensor work: one TF32 product per contraction, three for split-TF32; the TF32
            # dense peak is taken as half the measured BF16 GEMM rate (nominal 1:2 ratio)
            passes = 3 if math == "3xtf32" else 1
            tf32_peak = _bf16_peak() / 2
            out["tensor_tflops"] = out["tflops"] * passes
            out["tensor_frac_of_tf32_peak"] = out["tensor_tflops"] / tf32_peak
            out["tf32_peak_tflops"] = tf32_peak
        if dt == "f64":
            out["alu_frac_of_fp64_fma_rate"] = out["tflops"] / 2 * 1e3 / fma
    if blk == "line" and dt == "f64":
        # FP64 pipe roof: 7 operations per cell (6 for Gauss-Seidel with omega = 1, whose
        # update is the solve itself)
        ops = 6 if meth == "gs" else 7
        out["fp64_ops_per_cell"] = ops
        out["alu_frac_of_fp64_fma_rate"] = rate * ops / fma
    if dt == "f64":
        out["fp64_fma_rate_g"] = fma
    if not _NO_CPU_LEGS["on"]:
        # the x-sine form runs in calls of several sweeps: check such a call
        out["err_vs_oracle"], out["cpu_baseline"] = _grid_cpu_leg(
            brs, stream, blk, meth, dt, a, math, box, nsweeps=max(3, mmin) if modes else 1)
    return out


def _patch_views(arr, dims):
    import numpy as np

    offs = np.concatenate([[0], np.cumsum(np.asarray(dims).prod(axis=1))])
    return [arr[offs[q]:offs[q + 1]].reshape(int(d[2]), int(d[1]), int(d[0]))
            for q, d in enumerate(dims)]


def _batched_cpu_leg(brs, stream, dims, u0_np, b_np, dt="f32", sweeps=3, sample=12):
    """Chaotic batched GS: per sampled patch, the GPU residual after each of `sweeps`
    sweeps against the oracle's Jacobi (omega = 1) and ordered GS on that patch alone."""
    import numpy as np
    import torch

    orc = _orc()
    td = torch.float64 if dt == "f64" else torch.float32
    rng = np.random.default_rng(23)
    qs = sorted(set(int(q) for q in rng.choice(len(dims), sample, replace=False)) | {0})
    a = COEFFS
    ut = torch.from_numpy(u0_np).to(td).cuda()
    bt = torch.from_numpy(b_np).to(td).cuda()
    u0r = ut.double().cpu().numpy()
    br = bt.double().cpu().numpy()
    got = {q: [] for q in qs}
    with brs.BatchedContext(dims, a, method="gs", dtype=dt) as bc:
        for _ in range(sweeps):
            bc.sweep(ut, bt, 1, stream=stream)
            uv = _patch_views(ut.double().cpu().numpy(), dims)
            bv = _patch_views(br, dims)
            for q in qs:
                got[q].append(orc.residual_norm(uv[q], bv[q], a))
    worst_hi, worst_lo, cells, t0 = 0.0, 1e30, 0, time.perf_counter()
    uv0, bv = _patch_views(u0r, dims), _patch_views(br, dims)
    for q in qs:
        ref = {}
        for m in ("jacobi", "gs_lex", "gs_zebra", "gs_reverse"):
            u, rs = uv0[q], []
            for _ in range(sweeps):
                u = orc.sweep(u, bv[q], a, block="line", method=m, omega=1.0)
                rs.append(orc.residual_norm(u, bv[q], a))
            ref[m] = np.array(rs)
            cells += sweeps * u.size
        g = np.array(got[q])
        lo = np.minimum(np.minimum(ref["gs_lex"], ref["gs_zebra"]), ref["gs_reverse"])
        worst_hi = max(worst_hi, float(np.max(g / ref["jacobi"])))
        worst_lo = min(worst_lo, float(np.min(g / lo)))
    secs = time.perf_counter() - t0
    return ({"metric": "residual bracket of chaotic GS per sampled patch (not reproducible "
                       "element by element)", "patches_sampled": len(qs), "sweeps": sweeps,
             "max_ratio_to_jacobi_omega1": worst_hi, "min_ratio_to_best_ordered_gs": worst_lo,
             "within_bracket": worst_hi <= 1.1 and worst_lo >= 0.9},
            {"value": cells / secs / 1e9, "unit": UNIT, "cores": orc.num_threads(),
             "kind": "oracle",
             "sample": f"oracle Jacobi and three ordered line-GS sweeps x{sweeps} on "
                       f"{len(qs)} sampled patches, one patch after another ({secs:.2f} s)"})


def _batched_vs_fp64(brs, stream, dims, u0_np, b_np, sweeps=1000):
    """The batched FP32 form against the plain FP64 sweep at equal final residual: the same
    number of chaotic line-GS sweeps on every patch by (a) the batched FP32 graph launch,
    (b) the batched FP64 launch and (c) one FP64 single-grid context per patch (per-patch
    launches); final ||b - A u|| / ||b|| over all patches in FP64 for each."""
    import math

    import torch

    def rel_residual(u64, b64):
        tot, nb = 0.0, float(torch.linalg.norm(b64)) ** 2
        for (nx, ny, nz), uq, bq in zip(dims, _patch_views(u64, dims), _patch_views(b64, dims)):
            with brs.Context(int(nx), int(ny), int(nz), COEFFS, method="gs", dtype="f64") as c:
                tot += c.residual(uq.reshape(-1), bq.reshape(-1)) ** 2
        return math.sqrt(tot / nb)

    b64 = torch.from_numpy(b_np).cuda()
    out = {"sweeps": sweeps}
    for name, dt in (("batched_f32", "f32"), ("batched_f64", "f64")):
        td = torch.float64 if dt == "f64" else torch.float32
        u = torch.from_numpy(u0_np).to(td).cuda()
        bt = b64.to(td)
        with brs.BatchedContext(dims, COEFFS, method="gs", dtype=dt) as bc:
            bc.sweep(u, bt, 1, stream=stream)  # tune / capture outside the clock
            u.copy_(torch.from_numpy(u0_np).to(td))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            bc.sweep(u, bt, sweeps, stream=stream)
            torch.cuda.synchronize()
            out[name] = {"s": time.perf_counter() - t0,
                         "rel_residual": rel_residual(u.double(), b64)}
    ctxs = [brs.Context(int(nx), int(ny), int(nz), COEFFS, method="gs", dtype="f64")
            for nx, ny, nz in dims]
    u = torch.from_numpy(u0_np).cuda()
    views = list(zip(_patch_views(u, dims), _patch_views(b64, dims)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c, (uq, bq) in zip(ctxs, views):
        c.sweep(uq.reshape(-1), bq.reshape(-1), sweeps, stream=stream)
    torch.cuda.synchronize()
    out["plain_f64_per_patch"] = {"s": time.perf_counter() - t0,
                                  "rel_residual": rel_residual(u, b64)}
    for c in ctxs:
        c.close()
    out["speedup_batched_f32_vs_plain_f64"] = (out["plain_f64_per_patch"]["s"]
                                               / out["batched_f32"]["s"])
    return out


def _variant_batched(brs, stream, barrier, per_patch=True):
    """600 patches, dims from {16,24,32,48,64}, FP32 chaotic line GS, 20 sweeps."""
    import numpy as np
    import torch

    from brs_inputs import batched_fields, batched_patch_dims

    dims = batched_patch_dims(600)
    u0_np = batched_fields(dims, 2)
    b_np = batched_fields(dims, 1, scale_h2=True)
    u0 = torch.from_numpy(u0_np).float().cuda()
    b = torch.from_numpy(b_np).float().cuda()
    cells = int(u0.numel())
    with brs.BatchedContext(dims, COEFFS, method="gs", dtype="f32") as bc:
        cfg = bc.config()
        u = u0.clone()
        ms = _time_sweeps(bc, u, b, 5, 2, 20, stream, barrier)
    graph_rate = _rate(cells, 20 * 5, ms)
    out = {"workload": "batched600", "block": "line", "method": "gs", "dtype": "f32",
           "patches": 600, "cells": cells, "sweeps": 20, "value": graph_rate, "unit": UNIT,
           "hbm_frac": graph_rate * 12 / _peaks()[0], "tuned": cfg}
    if not per_patch:
        return out
    # per-patch launches of the single-grid path on the same data
    ctxs = [brs.Context(int(nx), int(ny), int(nz), COEFFS, method="gs", dtype="f32")
            for nx, ny, nz in dims]
    offs = np.concatenate([[0], np.cumsum(dims.prod(axis=1))])
    u = u0.clone()
    views = [(u[offs[q]:offs[q + 1]], b[offs[q]:offs[q + 1]]) for q in range(600)]
    for c, (uq, bq) in zip(ctxs, views):
        c.sweep(uq, bq, 1, stream=stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for c, (uq, bq) in zip(ctxs, views):
        c.sweep(uq, bq, 20, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    per_patch_rate = _rate(cells, 20, e0.elapsed_time(e1))
    for c in ctxs:
        c.close()
    out["per_patch_launches_value"] = per_patch_rate
    out["speedup_vs_per_patch"] = graph_rate / per_patch_rate
    out["vs_plain_fp64_equal_sweeps"] = _batched_vs_fp64(brs, stream, dims, u0_np, b_np)
    if not _NO_CPU_LEGS["on"]:
        out["err_vs_oracle"], out["cpu_baseline"] = _batched_cpu_leg(brs, stream, dims, u0_np,
                                                                     b_np)
    return out


def _level_cpu_leg(brs, stream, dims, nbr, u0_np, b_np, dt):
    """Level with ghost exchange, chaotic GS inside the patches: the GPU residual after one
    step against the oracle's level step with Jacobi (omega = 1) and lexicographic GS
    inside the patches (ghosts from before the step in both)."""
    import math

    import numpy as np
    import torch

    orc = _orc()
    td = torch.float64 if dt == "f64" else torch.float32
    u = torch.from_numpy(u0_np).to(td).cuda()
    bt = torch.from_numpy(b_np).to(td).cuda()
    u0r, br = u.double().cpu().numpy(), bt.double().cpu().numpy()
    with brs.BatchedContext(dims, COEFFS, method="gs", dtype=dt, nbr=nbr) as lc:
        lc.sweep(u, bt, 1, stream=stream)
        got = u.double().cpu().numpy()

    def level_res(v):
        # residual of the assembled level: each patch's own residual with the neighbours'
        # values as its ghosts (one oracle level step with omega = 0 leaves v unchanged and
        # so does not help); computed patch by patch with ghosts folded into b
        tot = 0.0
        offs = orc.level_offsets(dims)
        for q, (nx, ny, nz) in enumerate(dims):
            n = int(nx) * int(ny) * int(nz)
            vq = v[offs[q]:offs[q] + n].reshape(int(nz), int(ny), int(nx))
            bq = br[offs[q]:offs[q] + n].reshape(int(nz), int(ny), int(nx)).copy()
            for f in range(6):
                p2 = int(nbr[q][f])
                if p2 < 0:
                    continue
                n2 = int(np.prod(dims[p2]))
                w = v[offs[p2]:offs[p2] + n2].reshape(int(dims[p2][2]), int(dims[p2][1]),
                                                     int(dims[p2][0]))
                ax = f >> 1
                arr_ax = 2 - ax
                src = np.take(w, [-1] if f % 2 == 0 else [0], axis=arr_ax)
                dst = [slice(None)] * 3
                dst[arr_ax] = slice(0, 1) if f % 2 == 0 else slice(-1, None)
                bq[tuple(dst)] += COEFFS[ax] * src
            tot += orc.residual_norm(vq, bq, COEFFS) ** 2
        return math.sqrt(tot)

    t0 = time.perf_counter()
    rj = level_res(orc.level_sweep(u0r, br, dims, nbr, COEFFS, method="jacobi", omega=1.0))
    rl = level_res(orc.level_sweep(u0r, br, dims, nbr, COEFFS, method="gs_lex", omega=1.0))
    secs = time.perf_counter() - t0
    rg = level_res(got)
    return ({"metric": "residual bracket of one level step (chaotic GS inside the patches, "
                       "not reproducible element by element)",
             "ratio_to_jacobi_omega1": rg / rj, "ratio_to_lexicographic_gs": rg / rl,
             "within_bracket": rg <= 1.1 * rj and rg >= 0.9 * rl},
            {"value": 2 * u0r.size / secs / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
             "sample": f"two oracle level steps (Jacobi omega = 1, lexicographic GS) over all "
                       f"{len(dims)} patches with their residuals, {secs:.1f} s"})


def _variant_level(brs, stream, barrier, which, dt="f32"):
    """A level of patches with ghost exchange after every step (Sec. 2), chaotic x-line GS,
    3 steps per call (the paper's 3 smoothing steps): 96 x 64^3 as a 4 x 4 x 6 array, or the
    mixed 80-patch set of Table 2.  The same patches without the exchange give its share."""
    import torch

    from brs_inputs import batched_fields, level_tiling, table2_mixed_level

    if which == "level96x64":
        dims, nbr = level_tiling((4, 4, 6), (64, 64, 64))
    else:
        dims, nbr = table2_mixed_level()
    td = torch.float64 if dt == "f64" else torch.float32
    u0_np = batched_fields(dims, 2)
    b_np = batched_fields(dims, 1, scale_h2=True)
    u0 = torch.from_numpy(u0_np).to(td).cuda()
    b = torch.from_numpy(b_np).to(td).cuda()
    cells = int(u0.numel())
    steps = 10 if dt == "f32" else 2
    with brs.BatchedContext(dims, COEFFS, method="gs", dtype=dt, nbr=nbr) as lc:
        u = u0.clone()
        ms_gather = _time_sweeps(lc, u, b, steps, 2, 3, stream, barrier)
    # the calls only ever see the iterate the previous call left: ghosts kept across calls
    with brs.BatchedContext(dims, COEFFS, method="gs", dtype=dt, nbr=nbr) as lc:
        lc.keep_ghosts(True)
        u = u0.clone()
        ms = _time_sweeps(lc, u, b, steps, 2, 3, stream, barrier)
    with brs.BatchedContext(dims, COEFFS, method="gs", dtype=dt) as bc:
        u = u0.clone()
        ms0 = _time_sweeps(bc, u, b, steps, 2, 3, stream, barrier)
    rate = _rate(cells, 3 * steps, ms)
    es = 8 if dt == "f64" else 4
    out = {"workload": which, "block": "line", "method": "gs", "dtype": dt,
           "patches": int(len(dims)), "cells": cells, "sweeps_per_call": 3, "value": rate,
           "unit": UNIT, "hbm_frac": rate * 3 * es / _peaks()[0],
           "ghosts": "kept across calls (brsmooth_level_keep_ghosts)",
           "gather_per_call_value": _rate(cells, 3 * steps, ms_gather),
           "without_exchange_value": _rate(cells, 3 * steps, ms0),
           "ghost_exchange_share": max(0.0, (ms - ms0) / ms)}
    if not _NO_CPU_LEGS["on"]:
        out["err_vs_oracle"], out["cpu_baseline"] = _level_cpu_leg(brs, stream, dims, nbr,
                                                                   u0_np, b_np, dt)
    return out


FP64_CALL_SWEEPS = 1000  # plain FP64 plane Jacobi at 512^3: sweeps per call (residual between)


def _fp64_plane_solve(brs, b, a, rtol=1e-10, max_sweeps=40000):
    """Plain FP64 plane Jacobi (omega = 0.8) from u = 0 in calls of FP64_CALL_SWEEPS sweeps,
    the FP64 residual after each call, until ||r|| / ||b|| <= rtol: measured wall time."""
    import torch

    n = b.shape[0]
    nb = float(torch.linalg.norm(b))
    with brs.Context(n, n, n, a, block="plane", method="jacobi", dtype="f64") as o64:
        u = torch.zeros_like(b)
        o64.sweep(u, b, 2)  # warm-up (set-up of the tables and maps)
        u.zero_()
        sweeps, r, hist = 0, 1.0, []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while r > rtol and sweeps < max_sweeps:
            o64.sweep(u, b, FP64_CALL_SWEEPS)
            sweeps += FP64_CALL_SWEEPS
            r = o64.residual(u, b) / nb
            hist.append(r)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        if o64.last_error() != 0:
            raise RuntimeError("device status raised during the FP64 solve")
    return u, {"sweeps": sweeps, "sweeps_per_call": FP64_CALL_SWEEPS, "rel_residual": r,
               "s_measured": t, "residual_per_call": hist}


def _variant_defect512_fp64(brs, stream):
    """512^3, a=(1,0.1,0.01): the plain FP64 plane-Jacobi solve to ||r||/||b|| <= 1e-10 alone,
    and its distance to the oracle's exact solution."""
    import torch

    from brs_inputs import rhs

    a = (1.0, 0.1, 0.01)
    b_np = rhs((512, 512, 512))
    u, rec = _fp64_plane_solve(brs, torch.from_numpy(b_np).cuda(), a)
    out = {"workload": "grid512_aniso plain FP64 plane Jacobi to 1e-10", "coeffs": a, **rec}
    out["err_vs_oracle"], out["cpu_baseline"] = _defect_cpu_leg(b_np, a, u.cpu().numpy(),
                                                                rec["rel_residual"])
    return out


def _variant_defect(brs, stream):
    """512^3, a=(1,0.1,0.01): FP32 plane sweeps inside FP64 defect correction vs plain FP64
    plane Jacobi.  The inner sweeps (block Jacobi, omega = 0.8, or two-colour block GS,
    omega = 1; split-TF32 or single-TF32 products) and their count per outer step m are
    chosen by timed full solves on 64^3
    (where the plain FP64 solve is measured too); at 512^3 the mixed solve and the plain FP64
    plane-Jacobi solve (about 9000 sweeps) both run to ||r||/||b|| <= 1e-10 and are compared
    with the oracle's exact solution."""
    import torch

    from brs_inputs import rhs

    a = (1.0, 0.1, 0.01)
    out = {"workload": "grid512_aniso defect correction", "coeffs": a, "rtol": 1e-10}
    n = 64
    b = torch.from_numpy(rhs((n, n, n))).cuda()
    per = {}
    with brs.Context(n, n, n, a, block="plane", method="jacobi", dtype="f64") as o64:
        for meth, arith in ((mm, pm) for mm in ("jacobi", "gs") for pm in ("3xtf32", "tf32")):
            with brs.Context(n, n, n, a, block="plane", method=meth, dtype="f32",
                             plane_math=arith) as i32:
                # full solves to 1e-10 for m in {8, 32, 128}; the fastest (method, products,
                # m) is kept (a measured choice) and used at 512^3 below
                for m in (8, 32, 128):
                    u = torch.zeros_like(b)
                    brs.defect_correction(o64, i32, u, b, rtol=1e-10, inner_sweeps=m,
                                          max_outer=500)
                    u.zero_()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    d_m, r_m, _ = brs.defect_correction(o64, i32, u, b, rtol=1e-10,
                                                        inner_sweeps=m, max_outer=500)
                    per[f"{meth}_{arith}_m{m}"] = {"inner": meth, "math": arith, "m": m,
                                                  "outer": d_m,
                                           "inner_sweeps": d_m * m, "rel_residual": r_m,
                                           "s": time.perf_counter() - t0, "u": u.clone()}
        best = min(per, key=lambda k: per[k]["s"])
        best_meth, best_m, best_math = per[best]["inner"], per[best]["m"], per[best]["math"]
        u64 = torch.zeros_like(b)
        sweeps, r = 0, 1.0
        nb = float(torch.linalg.norm(b))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while r > 1e-10 and sweeps < 20000:
            o64.sweep(u64, b, 16)
            sweeps += 16
            r = o64.residual(u64, b) / nb
        t_f64 = time.perf_counter() - t0
    ustar = _orc().exact_solve(b.cpu().numpy(), a)
    errs = {"mixed": _rel_err(per[best]["u"].cpu().numpy(), ustar),
            "fp64": _rel_err(u64.cpu().numpy(), ustar)}
    for v in per.values():
        del v["u"]
    out["grid64_full_solve"] = {"err_vs_oracle_exact_rel_max": errs, "inner": best_meth,
                                "inner_products": best_math,
                                "inner_sweeps_m": best_m, "per_choice": per,
                                "mixed_outer": per[best]["outer"],
                                "mixed_inner_sweeps": per[best]["inner_sweeps"],
                                "mixed_rel_residual": per[best]["rel_residual"],
                                "mixed_s": per[best]["s"], "fp64_sweeps": sweeps,
                                "fp64_rel_residual": r, "fp64_s": t_f64}
    # 512^3: the mixed solve and the plain FP64 solve, each run to ||r|| / ||b|| <= 1e-10
    # (measured) and compared with the oracle's exact solution
    n = 512
    b_np = rhs((n, n, n))
    b = torch.from_numpy(b_np).cuda()
    with brs.Context(n, n, n, a, block="plane", method="jacobi", dtype="f64") as o64, \
            brs.Context(n, n, n, a, block="plane", method=best_meth, dtype="f32",
                        plane_math=best_math) as i32:
        u = torch.zeros_like(b)
        brs.defect_correction(o64, i32, u, b, rtol=0.0, inner_sweeps=best_m, max_outer=1)
        u.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done, rel, hist = brs.defect_correction(o64, i32, u, b, rtol=1e-10,
                                                inner_sweeps=best_m, max_outer=2000)
        torch.cuda.synchronize()
        t_mixed = time.perf_counter() - t0
        u_gpu = u.cpu().numpy()
        del u
    # the plain FP64 plane-Jacobi solve to the same residual, run in full
    u64, f64 = _fp64_plane_solve(brs, b, a)
    u64_np = u64.cpu().numpy()
    del u64
    import math

    # contraction per sweep of plane Jacobi (omega=0.8) on the slowest mode: g_111
    s1 = 2 - 2 * math.cos(math.pi / (n + 1))
    lam = (a[0] + a[1] + a[2]) * s1
    mu = a[0] * s1 + a[1] * s1 + 2 * a[2]
    g = 1 - 0.8 * lam / mu
    sweeps_needed = math.log(1e-10) / math.log(g)
    out["grid512"] = {"inner": best_meth, "inner_products": best_math, "inner_sweeps_m": best_m,
                      "mixed_s_measured": t_mixed,
                      "mixed_outer": done, "mixed_inner_sweeps": done * best_m,
                      "mixed_rel_residual": rel,
                      "fp64_plane_jacobi": f64,
                      "fp64_s_measured": f64["s_measured"],
                      "speedup_mixed_vs_fp64_measured": f64["s_measured"] / t_mixed,
                      "fp64_sweeps_slowest_mode_bound": sweeps_needed,
                      "note": "both arms measured to ||r||/||b|| <= 1e-10 (wall time of the "
                              "whole solve); the FP64 arm checks its residual after every "
                              "call of fp64_plane_jacobi.sweeps_per_call sweeps"}
    out["grid512"]["err_vs_oracle"], out["grid512"]["cpu_baseline"], fp64_err = _defect_cpu_leg(
        b_np, a, u_gpu, rel, also=(u64_np, f64["rel_residual"]))
    out["grid512"]["fp64_plane_jacobi"]["err_vs_oracle"] = fp64_err
    return out


def _defect_cpu_leg(b_np, a, u_gpu, rel, also=None):
    """512^3: the oracle's exact solution u* = A^-1 b (3D DST-I), timed, and the solve's
    distance to it.  With ||b - A u|| <= rel ||b|| the error obeys
    ||u - u*|| <= kappa(A) rel ||u*|| in the 2-norm.  also = (u, rel) of a second solve of
    the same problem: its distance is returned as a third item."""
    import math

    import numpy as np

    orc = _orc()
    n = b_np.shape[0]
    t0 = time.perf_counter()
    ustar = orc.exact_solve(b_np, a)
    secs = time.perf_counter() - t0
    s1 = 2 - 2 * math.cos(math.pi / (n + 1))
    sn = 2 - 2 * math.cos(n * math.pi / (n + 1))
    kappa = sum(a) * sn / (sum(a) * s1)

    def dist(u, r):
        d = u - ustar
        return {"metric": "distance of the final iterate to the oracle's exact DST solution",
                "rel_max_norm": float(np.max(np.abs(d)) / np.max(np.abs(ustar))),
                "rel_2norm": float(np.linalg.norm(d) / np.linalg.norm(ustar)),
                "bound_rel_2norm": kappa * r, "kappa_A": kappa}

    out = (dist(u_gpu, rel),
           {"value": b_np.size / secs / 1e9, "unit": "Gcell/s (exact solve)",
            "cores": orc.num_threads(), "kind": "oracle",
            "sample": f"the oracle's exact solve of the 512^3 problem (3D DST-I, scipy), "
                      f"{secs:.1f} s"})
    return out + (dist(*also),) if also is not None else out


STUDY_BLOCKS = [("box", (1, 1, 1)), ("box", (2, 2, 2)), ("box", (4, 2, 2)), ("box", (4, 4, 2)),
                ("box", (4, 4, 4)), ("box", (8, 4, 4)), ("box", (8, 8, 4)), ("box", (8, 8, 8)),
                ("line", (0, 0, 0)), ("plane", (0, 0, 0))]


def _variant_block_study(brs, stream, n=64, i_win=5000, k_win=100):
    """Sec. 3 block-size study on the paper's 64^3 patch, FP64, a=(1,1,1), b=0 and a random
    initial guess: ||r_3||/||r_0||, the sliding-window factor (||r_{i+k}||/||r_i||)^(1/k) at
    i = 5000, the time per sweep, and the time per decade of residual reduction.  For
    Jacobi with point, x-line and xy-plane blocks the asymptotic factor has a closed form
    (the slowest sine mode), reported beside the measurement."""
    import math

    import numpy as np
    import torch

    from brs_inputs import initial_guess

    a = (1.0, 1.0, 1.0)
    u0 = torch.from_numpy(initial_guess((n, n, n))).cuda()
    b = torch.zeros_like(u0)
    s1 = 2 - 2 * math.cos(math.pi / (n + 1))
    lam = 3 * s1
    closed = {"box(1, 1, 1)": 1 - 0.8 * lam / 6, "line": 1 - 0.8 * lam / (s1 + 4),
              "plane": 1 - 0.8 * lam / (2 * s1 + 2)}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    rows = []
    for blk, box in STUDY_BLOCKS:
        label = f"box{box}" if blk == "box" else blk
        for meth in ("jacobi", "gs"):
            with brs.Context(n, n, n, a, block=blk, method=meth, dtype="f64", box=box) as c:
                u = u0.clone()
                r0 = c.residual(u, b)
                c.sweep(u, b, 3)
                r3 = c.residual(u, b)
                torch.cuda.synchronize()
                e0.record(stream)
                c.sweep(u, b, i_win - 3)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / (i_win - 3)
                ri = c.residual(u, b)
                c.sweep(u, b, k_win)
                rk = c.residual(u, b)
                fac = (rk / ri) ** (1.0 / k_win) if ri > 0 and rk > 0 else None
                row = {"block": label, "method": meth, "r3_over_r0": r3 / r0,
                       "factor_at_5000": fac, "ms_per_sweep": ms,
                       "ms_per_decade": (ms * math.log(10) / -math.log(fac)
                                         if fac and 0 < fac < 1 else None)}
                if meth == "jacobi" and label in closed:
                    row["factor_closed_form"] = closed[label]
                rows.append(row)
    # oracle leg: ||r_3|| / ||r_0|| of every row from the oracle's own sweeps (the GPU's
    # Gauss-Seidel forms here all visit their blocks in two colours: the oracle's zebra)
    orc = _orc()
    u0n = u0.cpu().numpy()
    bn = np.zeros_like(u0n)
    r0 = orc.residual_norm(u0n, bn, a)
    t0 = time.perf_counter()
    worst = 0.0
    for row, (blk, box) in zip(rows, [bb for bb in STUDY_BLOCKS for _ in (0, 1)]):
        m = "jacobi" if row["method"] == "jacobi" else "gs_zebra"
        om = 0.8 if m == "jacobi" else 1.0
        v = u0n
        for _ in range(3):
            v = _orc_sweep(orc, v, bn, a, blk, box, m, om)
        row["r3_over_r0_oracle"] = orc.residual_norm(v, bn, a) / r0
        worst = max(worst, abs(row["r3_over_r0"] / row["r3_over_r0_oracle"] - 1.0))
    secs = time.perf_counter() - t0
    return {"workload": f"block_study {n}^3 FP64, a=(1,1,1), b=0, random initial guess",
            "window": {"i": i_win, "k": k_win}, "results": rows,
            "err_vs_oracle": {"metric": "largest relative difference of ||r_3||/||r_0|| "
                                        "between the GPU and the oracle over all rows",
                              "value": worst, "tolerance": 1e-10},
            "cpu_baseline": {"value": len(rows) * 3 * n ** 3 / secs / 1e9, "unit": UNIT,
                             "cores": orc.num_threads(), "kind": "oracle",
                             "sample": f"3 oracle sweeps of every row at {n}^3, {secs:.1f} s"}}


def _adjoint_cpu_leg(n, dt, b, u0, ut, grads):
    """Gradients against the oracle's FP64 reverse mode.  128^3: the whole grid.  384^3:
    dL/du0 and dL/db on sampled x-lines, each from the oracle run on the sub-grid of lines
    within distance 16 (8 sweeps forward and 8 back reach at most 16 lines: cut edges never
    reach the sampled line); the coefficient gradients are sums over the whole grid and
    are compared at 128^3."""
    import numpy as np

    orc = _orc()
    a = COEFFS
    gu, gb, ga = grads
    t0 = time.perf_counter()
    if n <= 128:
        _, gur, gbr, gar = orc.adjoint_gradients(u0, b, a, 8, ut, block="line", omega=0.8)
        secs = time.perf_counter() - t0
        err = {"metric": "relative max-norm over the whole grid",
               "dL_du0": _rel_err(gu, gur), "dL_db": _rel_err(gb, gbr),
               "dL_da_rel": float(np.max(np.abs(ga - gar) / np.abs(gar)))}
        cells = u0.size
        sample = f"oracle forward + reverse sweeps on the whole {n}^3 grid, {secs:.1f} s"
    else:
        R = 16
        picks = [(0, 0), (n // 2, n // 3), (n - 1, n // 2)]
        wu = wb = 0.0
        cells = 0
        for (j, k) in picks:
            j0, j1, k0, k1 = max(0, j - R), min(n, j + R + 1), max(0, k - R), min(n, k + R + 1)
            sl = (slice(k0, k1), slice(j0, j1))
            _, gur, gbr, _ = orc.adjoint_gradients(
                np.ascontiguousarray(u0[sl]), np.ascontiguousarray(b[sl]), a, 8,
                np.ascontiguousarray(ut[sl]), block="line", omega=0.8)
            wu = max(wu, _rel_err(gu[k, j], gur[k - k0, j - j0]))
            wb = max(wb, _rel_err(gb[k, j], gbr[k - k0, j - j0]))
            cells += gur.size
        secs = time.perf_counter() - t0
        err = {"metric": "relative max-norm on 3 sampled x-lines (sub-grids of radius 16)",
               "dL_du0": wu, "dL_db": wb}
        sample = f"oracle forward + reverse sweeps on 3 sub-grids of 33 x 33 lines, {secs:.1f} s"
    err["tolerance"] = 1e-11 if dt in ("f64", "float64") else 2e-5
    return err, {"value": 2 * 8 * cells / secs / 1e9, "unit": "Gcell-updates/s (fwd+bwd)",
                 "cores": orc.num_threads(), "kind": "oracle", "sample": sample}


def _variant_adjoint(brs, stream):
    """128^3 and 384^3, FP64 and FP32: 8 x-line Jacobi sweeps forward + adjoint backward
    (checkpoint every 4), loss 0.5 ||u_8 - u_t||^2, u_t ~ U[-1,1] (seed 3)."""
    import numpy as np
    import torch

    from brs_inputs import SEED_TARGET, initial_guess, rhs, uniform_field

    res = []
    for n, dt in ((128, torch.float64), (128, torch.float32), (384, torch.float64),
                  (384, torch.float32)):
        shape = (n, n, n)
        u0n, bn, utn = initial_guess(shape), rhs(shape), uniform_field(shape, SEED_TARGET)
        if dt == torch.float32:
            u0n = u0n.astype(np.float32).astype(np.float64)
            bn = bn.astype(np.float32).astype(np.float64)
        b = torch.from_numpy(bn).to(dt).cuda()
        u0 = torch.from_numpy(u0n).to(dt).cuda()
        ut = torch.from_numpy(utn).cuda()
        times = []
        for rep in range(3):
            bt = b.clone().requires_grad_(True)
            u0t = u0.clone().requires_grad_(True)
            at = torch.tensor(COEFFS, dtype=torch.float64, device="cuda", requires_grad=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            u = brs.block_smooth(bt, u0t, at, 8, ckpt=4)
            d = u.double() - ut
            (0.5 * (d * d).sum()).backward()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        best = min(times[1:])
        grads = (u0t.grad.double().cpu().numpy(), bt.grad.double().cpu().numpy(),
                 at.grad.cpu().numpy())
        del bt, u0t, u, d
        row = {"n": n, "dtype": str(dt).replace("torch.", ""), "sweeps": 8, "ckpt": 4,
               "fwd_bwd_s": best, "value": n ** 3 * 8 / best / 1e9,
               "unit": "Gcell-updates/s (fwd+bwd)"}
        if not _NO_CPU_LEGS["on"]:
            row["err_vs_oracle"], row["cpu_baseline"] = _adjoint_cpu_leg(n, row["dtype"], bn,
                                                                         u0n, utn, grads)
        res.append(row)
        del b, u0, ut
        torch.cuda.empty_cache()
    return {"workload": "adjoint", "results": res}


ISO, ANISO = (1.0, 1.0, 1.0), (1.0, 1.0, 0.01)


def _config2_matrix():
    """The 256^3 matrix of the config: {x-line, xy-plane} x {Jacobi, GS} x {FP64, FP32} x
    {a = (1,1,1), (1,1,0.01)} (FP64 x-line Jacobi at a = (1,1,1) is the headline);
    name -> (block, method, dtype, coeffs, steps, sweeps per step, plane math)."""
    out = {}
    for blk in ("line", "plane"):
        for a, tag in ((ISO, "iso"), (ANISO, "aniso")):
            for dt in ("f64", "f32"):
                for meth in ("jacobi", "gs"):
                    if (blk, meth, dt, a) == ("line", "jacobi", "f64", ISO):
                        continue
                    if blk == "line":
                        st, sw = (2, 50) if dt == "f64" else (6, 50)
                    else:
                        st, sw = (1, 50) if dt == "f64" else (4, 50)
                    out[f"{blk}_{meth}_{dt}_{tag}"] = (blk, meth, dt, a, st, sw, "auto")
    return out


VARIANTS = dict(_config2_matrix())
VARIANTS.update({
    # other arithmetic of the FP32 plane solve
    "plane_jacobi_f32_tf32_aniso": ("plane", "jacobi", "f32", ANISO, 4, 50, "tf32"),
    "plane_jacobi_f32_simt_aniso": ("plane", "jacobi", "f32", ANISO, 2, 50, "simt"),
    # the per-sweep form of the plane solve (two tensor-core products per sweep), which
    # calls of one or two sweeps run (BRSMOOTH_PLANE_MODES=0 below)
    "plane_jacobi_f32_aniso_per_sweep": ("plane", "jacobi", "f32", ANISO, 4, 10, "auto"),
    "plane_gs_f32_aniso_per_sweep": ("plane", "gs", "f32", ANISO, 4, 10, "auto"),
    "plane_jacobi_f32_tf32_aniso_per_sweep": ("plane", "jacobi", "f32", ANISO, 4, 10, "tf32"),
    "plane_jacobi_f64_aniso_per_sweep": ("plane", "jacobi", "f64", ANISO, 1, 2, "auto"),
    # y- and z-lines (x-line sweeps of the permuted grid; three grid passes per call)
    "yline_jacobi_f32": ("yline", "jacobi", "f32", (0.01, 1.0, 0.01), 6, 50, "auto"),
    "zline_jacobi_f32": ("zline", "jacobi", "f32", (0.01, 0.01, 1.0), 6, 50, "auto"),
    "zline_gs_f32": ("zline", "gs", "f32", (0.01, 0.01, 1.0), 6, 50, "auto"),
})
BOX_VARIANTS = {
    # name: (method, dtype, box, steps, sweeps per step, math); a = (1, 1, 1)
    "box_jacobi_f32_8cubed_3xtf32": ("jacobi", "f32", (8, 8, 8), 4, 10, "3xtf32"),
    "box_gs_f32_8cubed_3xtf32": ("gs", "f32", (8, 8, 8), 4, 10, "3xtf32"),
    "box_jacobi_f32_8cubed_tf32": ("jacobi", "f32", (8, 8, 8), 4, 10, "tf32"),
    "box_jacobi_f32_8cubed_simt": ("jacobi", "f32", (8, 8, 8), 2, 5, "simt"),
    "box_jacobi_f32_4cubed_3xtf32": ("jacobi", "f32", (4, 4, 4), 4, 10, "3xtf32"),
    "box_gs_f64_8cubed": ("gs", "f64", (8, 8, 8), 1, 2, "auto"),
    "box_gs_f64_4cubed": ("gs", "f64", (4, 4, 4), 1, 5, "auto"),
    # y- and z-lines as 1 x 256 x 1 and 1 x 1 x 256 boxes (dense inverse applied per line;
    # the line blocks themselves are the yline / zline variants)
    "box_jacobi_f32_yline_3xtf32": ("jacobi", "f32", (1, 256, 1), 4, 10, "3xtf32"),
    "box_jacobi_f32_zline_3xtf32": ("jacobi", "f32", (1, 1, 256), 4, 10, "3xtf32"),
}
SPECIAL = ("batched600", "level96x64", "table2_mixed", "level96x64_f64", "defect512", "adjoint",
           "block_study64")
PROFILE_ONLY = ("batched600_graph", "plane512_f32", "defect512_fp64")


# the headline workload as a named variant, for profiling runs (`--only`)
PROFILE_GRID = {"line_jacobi_f64_iso": ("line", "jacobi", "f64", ISO, 4, 50, "auto")}
_NO_CPU_LEGS = {"on": False}


def _variant_plane512(brs, stream, barrier, steps):
    """Plane Jacobi sweeps at 512^3, a = (1, 0.1, 0.01), FP32 split-TF32: the inner sweep of
    the 512^3 defect correction, timed alone (for profiling)."""
    import torch

    from brs_inputs import initial_guess, rhs

    n = 512
    a = (1.0, 0.1, 0.01)
    u = torch.from_numpy(initial_guess((n, n, n))).float().cuda()
    b = torch.from_numpy(rhs((n, n, n))).float().cuda()
    with brs.Context(n, n, n, a, block="plane", method="jacobi", dtype="f32") as c:
        ms = _time_sweeps(c, u, b, steps, 1, 2, stream, barrier)
    rate = _rate(n ** 3, 2 * steps, ms)
    return {"workload": "grid512_aniso plane Jacobi", "dtype": "f32", "plane_math": "3xtf32",
            "value": rate, "unit": UNIT, "ms_per_sweep": ms / (2 * steps),
            "tensor_frac_of_tf32_peak": rate * 4.0 * n * 3 / 1e3 / (_bf16_peak() / 2)}


def _run_variant(name, brs, stream, barrier, peak, steps=None):
    if name.endswith("_per_sweep"):
        # environment of the library's context set-up, restored afterwards
        old = os.environ.get("BRSMOOTH_PLANE_MODES")
        os.environ["BRSMOOTH_PLANE_MODES"] = "0"
        try:
            out = _run_variant_env(name, brs, stream, barrier, peak, steps)
        finally:
            if old is None:
                del os.environ["BRSMOOTH_PLANE_MODES"]
            else:
                os.environ["BRSMOOTH_PLANE_MODES"] = old
        out["plane_modes"] = "off (per-sweep form)"
        return out
    return _run_variant_env(name, brs, stream, barrier, peak, steps)


def _run_variant_env(name, brs, stream, barrier, peak, steps=None):
    if name == "batched600":
        return _variant_batched(brs, stream, barrier)
    if name == "batched600_graph":
        return _variant_batched(brs, stream, barrier, per_patch=False)
    if name == "plane512_f32":
        return _variant_plane512(brs, stream, barrier, steps or 3)
    if name in ("level96x64", "table2_mixed"):
        out = _variant_level(brs, stream, barrier, name)
        out["name"] = name
        return out
    if name == "level96x64_f64":
        out = _variant_level(brs, stream, barrier, "level96x64", "f64")
        out["name"] = name
        return out
    if name == "defect512":
        return _variant_defect(brs, stream)
    if name == "defect512_fp64":
        return _variant_defect512_fp64(brs, stream)
    if name == "adjoint":
        return _variant_adjoint(brs, stream)
    if name == "block_study64":
        return _variant_block_study(brs, stream)
    if name in BOX_VARIANTS:
        meth, dt, box, st, sw, math = BOX_VARIANTS[name]
        out = _variant_grid(brs, stream, barrier, peak, "box", meth, dt, COEFFS, steps or st, sw,
                            math, box)
        out["name"] = name
        return out
    blk, meth, dt, a, st, sw, math = VARIANTS[name] if name in VARIANTS else PROFILE_GRID[name]
    out = _variant_grid(brs, stream, barrier, peak, blk, meth, dt, a, steps or st, sw, math)
    out["name"] = name
    return out


def _variants(brs, stream, barrier, peak):
    out = []
    for name in list(VARIANTS) + list(BOX_VARIANTS) + list(SPECIAL):
        try:
            out.append(_run_variant(name, brs, stream, barrier, peak))
        except Exception as exc:  # report, do not hide
            out.append({"name": name, "error": repr(exc)})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--only", default=None,
                    help="run one named workload variant and print its JSON (for profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        import torch

        import paper_1208_1975_gb300 as brs

        brs.build()
        _NO_CPU_LEGS["on"] = args.no_cpu  # profiling runs: GPU work only
        res = _run_variant(args.only, brs, torch.cuda.current_stream(), None, _peaks()[0],
                           steps=args.steps)
        print(json.dumps(res), flush=True)
        return 0

    import torch

    import paper_1208_1975_gb300 as brs

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    barrier = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        barrier = dist.barrier
    if rank == 0:
        brs.build()
    if barrier:
        barrier()
    brs.lib()

    stream = torch.cuda.current_stream()
    cells = N * N * N
    u0, b_h = _inputs("f64")
    u = u0.cuda()
    b = b_h.cuda()
    ctx = brs.Context(N, N, N, COEFFS, block="line", method="jacobi", dtype="f64")

    sampler = ClockSampler(local)
    ms = _time_sweeps(ctx, u, b, args.steps, args.warmup, SWEEPS_PER_STEP, stream, barrier)
    clocks = sampler.stop()
    ms = max_over_ranks(ms, ws)
    sweeps_total = args.steps * SWEEPS_PER_STEP
    value = whole_job_rate(cells, sweeps_total, ms / 1e3, ws)

    # roofs of the sweep kernel: FP64 pipe operations (binding) and HBM bytes
    launch_ms = _launch_ms(ctx, u, b, stream)
    fma_rate = _live_fp64_fma_rate(brs, stream)
    ops_per_cell = 7  # gather 2 adds + 2 FMAs, one FMA per elimination direction, update FMA
    sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    smax = clocks.get("sm_max_mhz") or 2070.0
    alu_achieved = ops_per_cell * cells / (launch_ms / 1e3) / 1e9
    kernel = "xline_twist_kernel<false> (FP64 x-line Jacobi, omega = 0.8)"
    traffic = _traffic_record("line_twist_f64_256cubed.md", ["line_seq.cu", "brs_internal.cuh"])
    roofline = {"bound": "alu", "achieved": alu_achieved, "peak": fma_rate / 1e9,
                "unit": "GFP64op/s", "frac": alu_achieved / (fma_rate / 1e9),
                "traffic": traffic, "kernel": kernel, "ops_per_cell": ops_per_cell,
                "op": "one FP64 pipe instruction (FMA or ADD)",
                "launch_ms": launch_ms, "launches_per_step": SWEEPS_PER_STEP,
                "peak_source": "FP64 FMA probe kernel timed in this run (CUDA events)",
                "peak_derived": 2 * sm * smax / 1e3,
                "peak_derived_note": "2 FP64 FMA per clock per SM x SMs x max SM clock (GHz)"}
    peak, peak_kind = _peaks()
    hbm_achieved = 3 * 8 * cells / (launch_ms / 1e3) / 1e9
    live = _live_copy_gbs()
    roofline_hbm = {"bound": "hbm", "achieved": hbm_achieved, "peak": peak, "unit": "GB/s",
                    "frac": hbm_achieved / peak, "traffic": traffic, "kernel": kernel,
                    "alg_bytes_per_launch": 3 * 8 * cells, "live_copy_gbs": live,
                    "peak_source": f"{peak_kind} hbm_gbs"}

    # end to end through the host-buffer entry point (pinned host arrays): every step copies
    # its u and b in, sweeps, and copies u back.  Steps are independent problems, so they
    # alternate between two contexts on two streams and one step's copies overlap the
    # other's sweeps (the asynchronous host entry point); the clock stops once both streams
    # have drained.
    bh = b_h.pin_memory()
    uhs = [u0.pin_memory(), u0.clone().pin_memory()]
    streams = [stream, torch.cuda.Stream()]
    ctx2 = brs.Context(N, N, N, COEFFS, block="line", method="jacobi", dtype="f64")
    ctxs = [ctx, ctx2]
    e2e_steps = max(4, min(args.steps, 40))
    for q in range(4):
        ctxs[q % 2].sweep_host(uhs[q % 2], bh, SWEEPS_PER_STEP, stream=streams[q % 2],
                               wait=False)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for q in range(e2e_steps):
        ctxs[q % 2].sweep_host(uhs[q % 2], bh, SWEEPS_PER_STEP, stream=streams[q % 2],
                               wait=False)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    for cx in ctxs:
        if cx.last_error() != 0:
            raise RuntimeError("device status raised during the end-to-end steps")
    e2e_s = max_over_ranks(e2e_s, ws)
    e2e = {"value": whole_job_rate(cells, SWEEPS_PER_STEP * e2e_steps, e2e_s, ws), "unit": UNIT,
           "h2d_bytes_per_step": 2 * 8 * cells, "d2h_bytes_per_step": 8 * cells,
           "steps": e2e_steps,
           "timer": "host wall clock; steps alternate over two contexts and streams "
                    "(brsmooth_sweep_host_async), clock stopped after both streams drain"}
    ctx2.close()
    ctx.close()

    variants = []
    if not args.no_variants:
        variants = _variants(brs, stream, barrier, peak)

    if rank != 0:
        return 0
    cpu = None if args.no_cpu else _cpu_baseline()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "grid256_iso_f64: 256^3 x-line block Jacobi, a=(1,1,1), "
                                   "omega=0.8, FP64, b=h^2 f, f,u0 ~ U[-1,1] seeded",
                       "nx": N, "ny": N, "nz": N, "sweeps_per_step": SWEEPS_PER_STEP,
                       "parallelism": f"replicas x{ws}",
                       "l2": "inputs larger than L2: u, b and the line-major copies are "
                             "134 MB each (FP64) vs the 129 MB L2"},
            "gpu_launches": args.steps * (SWEEPS_PER_STEP + 3),
            "gpu_launches_note": "per step: 2 copies into the line-major layout, 50 sweeps, "
                                 "1 copy back",
            "roofline": roofline, "roofline_hbm": roofline_hbm, "cpu_baseline": cpu,
            "e2e": e2e, "clocks": clocks, "variants": variants}
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
