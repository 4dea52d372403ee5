"""Benchmark of the HOPE per-stage tendency on GB300.

Workload (default): C90 cubed sphere (6 x 90 x 90 cells), 11th-order TPP reconstruction
(11 x 11 stencil, 6 Gauss points per edge), FP64, steady geostrophic flow rotated by
alpha = pi/4 (with the matching tilted rotation axis), SSP-RK3 with dt = 300 s; one
benchmark step = one SSP-RK3 time step (three passes of the whole stage: ghost fill,
reconstruction + sources, LMARS fluxes + quadrature, tendency + RK combination) followed
by the FP64 mass diagnostic.  --steps defaults to 288 steps = one simulated day.

Metric: cell-stage updates per second (cells x stages / time), whole job.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica (the path has no data
exchange between spheres); timing takes the max over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CELLS, ORDER, DT = 90, 11, 300.0
ALPHA = np.pi / 4
WORKLOAD = "C90 TPP11 geostrophic alpha=pi/4, FP64, SSP-RK3 dt=300s"
METRIC = "cell-stage updates/s"
L2_FLUSH_BYTES = 512 << 20

# DRAM bytes per launch of the dominant kernel from the ncu capture summarised in
# profiles/recon_tpp11_c90_fp64.md (None until captured for the current kernel).
# DRAM bytes of one launch of the reconstruction from the last ncu capture
# (profiles/recon_tpp11_c90_fp64.md: 20.393728 MB read + 5.376 KB written).  The kernel has
# changed since (a griddepcontrol wait before its first access, memory accesses unchanged),
# so the line's `traffic` is null and the figure travels as `traffic_last_capture`.
RECON_TRAFFIC_BYTES = 20399104
RECON_TRAFFIC_CURRENT = False


def recon_flops_per_launch(N, K):
    """Algorithmic FLOPs of one TPP reconstruction + sources launch (one stage), the
    measurement plan's count (sum-factorised, each output point computed once): x-pass over
    N x (N + 2H) cells at me + 2 positions and y-pass at the n_poc = 4 me + me^2 points (K
    FMAs each, 3 variables), plus 28 flops of metric and Coriolis sources per cell point
    (eqs. 2.2, 2.3, with the point polynomials tabulated)."""
    me, H = (K + 1) // 2, (K - 1) // 2
    npoc = 4 * me + me * me
    per_panel = 3 * 2 * K * ((me + 2) * N * (N + 2 * H) + npoc * N * N) + 28 * me * me * N * N
    return 6 * per_panel


def recon_flops_evaluated_per_launch(N, K):
    """The FLOPs the kernel evaluates for the same outputs: the positions taken in mirror
    pairs (the weights at -xi are the weights at +xi reversed), per line K - 1 flops to fold
    it into sums and differences, 2K per pair (E: H + 1 terms, O: H terms, E +- O), K for
    the middle node of odd me; plus 28 flops of sources per cell point."""
    me, H = (K + 1) // 2, (K - 1) // 2
    gp, odd = me // 2, me % 2
    line_x = (K - 1) + (1 + gp) * 2 * K + odd * K            # the me + 2 x positions
    edge_col = (K - 1) + gp * 2 * K + odd * K                # west/east columns: me nodes
    node_col = (K - 1) + (1 + gp) * 2 * K + odd * K          # node columns: 2 edges + me nodes
    per_panel = 3 * (line_x * N * (N + 2 * H) + (2 * edge_col + me * node_col) * N * N) \
        + 28 * me * me * N * N
    return 6 * per_panel


# per edge point, LMARS of eqs. 3.30-3.38 as printed (a square root or division counts 1)
# plus the quadrature; the evaluated form (phi 2, the shared reciprocal 2, velocities 6,
# square roots 2, c 2, m* 4, phi* 5, m 1, the upwind flux m q_up 3, pressure 5, quadrature
# 6) takes 38
LMARS_FLOPS = 53
LMARS_FLOPS_EVALUATED = 38


def weno_recon_flops_per_launch(N, K):
    """Algorithmic FLOPs of one genuine-2D WENO reconstruction + sources launch, counted
    from the method's steps as the library evaluates them (FMA = 2): indicators of the
    L^2 sub-stencils through the factorised forms, tau and the weights f, the sub-stencil
    values at the n_poc points (x-pass per sub-stencil column, y-pass per row), the split
    combination, and 28 flops of sources per cell point."""
    L = (K + 1) // 2
    S, me = L * L, L
    npos, npoc = me + 2, 4 * me + me * me
    beta = L * L * (K * (L + 1) + L * L * (L + 2))
    tau = S * (S - 1) // 2 + 3 * S / 2
    points = npos * L * K * L + L * npoc * L * (L + 3)
    comb = npoc * (2 * S + 5) / 2
    per_cell = 3 * 2 * (beta + tau + points + comb) + 28 * me * me
    return 6 * N * N * per_cell


def weno1d_recon_flops_per_launch(N, K):
    """Algorithmic FLOPs of one dimension-by-dimension WENO-Z reconstruction + sources
    launch (section 5.5's comparator, FMA = 2, reciprocal = 1): per cell and variable, the
    indicators and factors of K stencil rows and NPOS row-value columns (L sub-stencils x L
    eigen-modes of 3 L + 3 flops, tau, f), and K NPOS + n_poc line values (L sub-stencil
    values and split sums of 2 L + 8 flops each, 7 for the combination); 28 flops of sources
    per cell point."""
    L = (K + 1) // 2
    me, npos, npoc = L, L + 2, 4 * L + L * L
    ind = L * L * (3 * L + 3) + 2 + 4 * L
    val = L * (2 * L + 8) + 7
    per_cell = 3 * ((K + npos) * ind + (K * npos + npoc) * val) + 28 * me * me
    return 6 * N * N * per_cell


def stage_flops(N, K, ghost_nnz, weno=False, evaluated=False):
    """Algorithmic FLOPs of one RK stage on one sphere: ghost fill (10 per nonzero of G),
    reconstruction + sources (TPP; weno=True: genuine-2D WENO; weno="1d": the
    dimension-by-dimension comparator), LMARS + quadrature at the 12 N^2 me edge points,
    tendency + stage combination (30 per cell).  evaluated=True: the TPP reconstruction and
    LMARS counted as the kernels evaluate them (mirror pairs, upwind flux)."""
    me = (K + 1) // 2
    if weno == "1d":
        rec = weno1d_recon_flops_per_launch(N, K)
    elif weno:
        rec = weno_recon_flops_per_launch(N, K)
    else:
        rec = recon_flops_evaluated_per_launch(N, K) if evaluated else recon_flops_per_launch(N, K)
    lm = LMARS_FLOPS_EVALUATED if evaluated else LMARS_FLOPS
    return 10 * ghost_nnz + rec + 12 * N * N * me * lm + 6 * N * N * 30


def roofline(flops_per_stage, stages_per_s, peak):
    a = flops_per_stage * stages_per_s
    return {"bound": "alu", "flops_per_stage": flops_per_stage, "achieved_tflops": a / 1e12,
            "peak_tflops": peak / 1e12, "frac": a / peak}


def measured_hbm_bps(default_gbs=6800.0):
    """Copy bandwidth of the GB300s (MEASURED_PEAKS.json beside this file), else the
    fallback figure; returns (bytes/s, source)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]) * 1e9, "measured"
    except (OSError, KeyError, ValueError):
        return default_gbs * 1e9, "fallback"


def step_roofline(flops_per_stage, state_bytes, g_bytes, stage_s, alu_peak, hbm_bps):
    """Whole-stage roofline, two ways: the state alone (q_stage and q^n read, q_next written)
    and the state plus one pass over the ghost operator streamed as a sparse matrix
    (nnz x (weight + index) bytes).  Roofline time = max(FLOPs / ALU peak, bytes / HBM);
    frac = roofline time / measured stage time."""
    out = {"flops_per_stage": flops_per_stage, "alu_peak_tflops": alu_peak / 1e12, "hbm_gbs": hbm_bps / 1e9}
    for name, b in (("state", state_bytes), ("state_plus_G", state_bytes + g_bytes)):
        t_alu, t_hbm = flops_per_stage / alu_peak, b / hbm_bps
        out[name] = {"bytes_per_stage": b, "bound": "alu" if t_alu >= t_hbm else "hbm",
                     "roofline_ms": 1e3 * max(t_alu, t_hbm), "frac": max(t_alu, t_hbm) / stage_s}
    return out


# panel frames (n, e1, e2) of the state layout: panel p maps (X, Y) to (n + X e1 + Y e2)/delta
PANEL_FRAMES = (((1, 0, 0), (0, 1, 0), (0, 0, 1)), ((0, 1, 0), (-1, 0, 0), (0, 0, 1)),
                ((-1, 0, 0), (0, -1, 0), (0, 0, 1)), ((0, -1, 0), (1, 0, 0), (0, 0, 1)),
                ((0, 0, 1), (0, 1, 0), (-1, 0, 0)), ((0, 0, -1), (0, 1, 0), (1, 0, 0)))


def cell_geometry(N):
    """Cell-centre longitude and latitude, and the cell average of the unit-sphere sqrtG
    (eq. 2.8 over r^2, 6-point Gauss rule per direction), each of shape (6, N, N)."""
    dx = np.pi / (2 * N)
    c = -np.pi / 4 + (np.arange(N) + 0.5) * dx
    X, Y = np.meshgrid(np.tan(c), np.tan(c), indexing="xy")  # [j][i]
    d = np.sqrt(1 + X * X + Y * Y)
    lon, lat = np.empty((6, N, N)), np.empty((6, N, N))
    for p, (n, e1, e2) in enumerate(PANEL_FRAMES):
        P = [(n[a] + X * e1[a] + Y * e2[a]) / d for a in range(3)]
        lon[p], lat[p] = np.arctan2(P[1], P[0]), np.arcsin(np.clip(P[2], -1, 1))
    g, w = np.polynomial.legendre.leggauss(6)
    xs = c[:, None] + 0.5 * dx * g[None, :]  # [cell][node]
    T = np.tan(xs)
    sq = (1 + T[None, :, None, :] ** 2) * (1 + T[:, None, :, None] ** 2)  # [j][i][gy][gx]
    sq = sq / (1 + T[None, :, None, :] ** 2 + T[:, None, :, None] ** 2) ** 1.5
    sg = np.einsum("jiyx,y,x->ji", sq, w / 2, w / 2)
    return lon, lat, np.broadcast_to(sg, (6, N, N)).copy()


def front_anisotropy(h, lon, lat, lon0, lat0, dcell, jump, dmax):
    """Azimuthal spread of a field about a centre (section 5.5's isotropy comparison):
    cells are binned by great-circle distance d (bins of half a cell up to dmax), the
    azimuthal mean profile hbar(d) is interpolated linearly between bin centres, and
      spread     = RMS over cells of (h - hbar(d)) / jump,
      axis_diag  = RMS over bins of the difference between the mean residuals h - hbar(d) of
                   the grid-axis sectors (azimuth within 10 degrees of 0, 90, 180, 270) and of
                   the diagonal sectors (45, 135, 225, 315), over jump.
    An isotropic field gives ~0 for both; a grid imprint shows in axis_diag."""
    h, lon, lat = (np.ravel(a) for a in (h, lon, lat))
    cd = np.sin(lat0) * np.sin(lat) + np.cos(lat0) * np.cos(lat) * np.cos(lon - lon0)
    dist = np.arccos(np.clip(cd, -1.0, 1.0))
    az = np.arctan2(np.sin(lon - lon0) * np.cos(lat),
                    np.cos(lat0) * np.sin(lat) - np.sin(lat0) * np.cos(lat) * np.cos(lon - lon0))
    sel = dist < dmax
    h, dist, az = h[sel], dist[sel], az[sel]
    bw = 0.5 * dcell
    nb = int(np.ceil(dmax / bw))
    b = np.minimum((dist / bw).astype(int), nb - 1)
    cnt = np.bincount(b, minlength=nb)
    ok = cnt >= 8
    mean = np.bincount(b, weights=h, minlength=nb)[ok] / cnt[ok]
    centre = np.bincount(b, weights=dist, minlength=nb)[ok] / cnt[ok]
    hbar = np.interp(dist, centre, mean)
    spread = float(np.sqrt(np.mean((h - hbar) ** 2)) / jump)
    sector = np.mod(np.degrees(az), 90.0)
    axis = (sector < 10.0) | (sector > 80.0)
    diag = np.abs(sector - 45.0) < 10.0

    r = h - hbar  # residual about the interpolated mean profile (removes each bin's own slope)

    def prof(m):
        c = np.bincount(b[m], minlength=nb)
        s = np.bincount(b[m], weights=r[m], minlength=nb)
        return c, s
    ca, sa = prof(axis)
    cg, sg = prof(diag)
    both = (ca >= 4) & (cg >= 4)
    diff = sa[both] / ca[both] - sg[both] / cg[both]
    axis_diag = float(np.sqrt(np.mean(diff ** 2)) / jump) if both.any() else float("nan")
    return {"spread": spread, "axis_diag": axis_diag, "bins": int(ok.sum())}


def cpu_model():
    """The host CPU's model line from /proc/cpuinfo (x86 'model name', Arm implementer/part)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return None
    for line in info:
        if line.lower().startswith("model name"):
            return line.split(":", 1)[1].strip()
    fields = {}
    for line in info:
        if ":" in line:
            k, v = (x.strip() for x in line.split(":", 1))
            fields.setdefault(k, v)
    if "CPU implementer" in fields or "CPU part" in fields:
        return "arm implementer %s part %s" % (fields.get("CPU implementer", "?"), fields.get("CPU part", "?"))
    return None


def set_host_threads(n):
    """Thread count of the OpenMP runtime the oracle uses (libgomp); False if unavailable."""
    import ctypes
    try:
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(int(n))
        return True
    except OSError:
        return False


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x, world, device="cuda"):
    """Max over ranks (the job's time is its slowest replica's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, cells, steps, seconds):
    """Whole-job cell-stage updates per second: every rank steps its own replica (weak
    scaling), the job takes the slowest rank's time."""
    return world * cells * 3 * steps / seconds


def _time_steps(s, q, dt, n, stream):
    """CUDA-event time of n graph-replayed steps on `stream` (after one warm-up step)."""
    import torch
    with torch.cuda.stream(stream):
        s.step(q, dt, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(q, dt, n)
        e1.record(stream)
        torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def _run(s, q, dt, n, stream):
    """CUDA-event milliseconds of one n-step run on `stream` (graphs captured beforehand
    by the caller's warm-up)."""
    import torch
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(q, dt, n)
        e1.record(stream)
        torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _rel(a, b):
    import torch
    return float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))


def measure_forms(hp, stream, fp64_peak):
    """The precision, differentiation and batching forms on the same box, each at the length
    its workload states, with its error (throughput in cell-stage updates/s)."""
    import torch
    from synth import bump_centres
    out = {}
    fp32_peak = hp.measure_fma_peak(hp.HOPE_FP32)
    out["fp32_fma_peak_tflops"] = fp32_peak / 1e12
    cells = 6 * N_CELLS * N_CELLS
    day = int(round(86400.0 / DT))
    # precision form on the headline workload: FP32 bulk path, one day against FP64
    s64 = hp.Sphere(N_CELLS, ORDER, hp.HOPE_TPP, hp.HOPE_FP64, coriolis_tilt=ALPHA)
    s = hp.Sphere(N_CELLS, ORDER, hp.HOPE_TPP, hp.HOPE_FP32, coriolis_tilt=ALPHA)
    qa = s64.geostrophic(ALPHA)
    q64, q32 = qa.clone(), qa.float().contiguous()
    m0 = s.mass(q32)
    with torch.cuda.stream(stream):
        s64.step(q64, DT, day)
        s.step(q32, DT, day)
    torch.cuda.synchronize()
    q = q32.clone()
    ms = _time_steps(s, q, DT, 100, stream)
    s.set_profiling(True)
    with torch.cuda.stream(stream):
        s.step(q, DT)
        rec = []
        ksum = np.zeros(4)
        for _ in range(20):
            s.step(q, DT)
            kt = s.kernel_times()
            rec.extend(st[1] for st in kt)
            ksum += np.sum(np.array(kt), axis=0)
    s.set_profiling(False)
    fl = recon_flops_per_launch(N_CELLS, ORDER)
    out["tpp11_c90_fp32"] = {"value": cells * 3 / (ms * 1e-3), "ms_per_step": ms,
                             "recon_ms": float(np.mean(rec)),
                             "stage_kernel_ms": dict(zip(("ghost", "recon", "flux", "update"), (ksum / 60).tolist())),
                             "recon_frac_of_fp32_peak": fl / (np.mean(rec) * 1e-3) / fp32_peak,
                             "days": day * DT / 86400.0,
                             "rel_l2_h_vs_fp64": _rel(q32[0], q64[0]),
                             "rel_l2_h_vs_analytic": _rel(q32[0], qa[0]),
                             "fp64_rel_l2_h_vs_analytic": _rel(q64[0], qa[0]),
                             "mass_drift": (s.mass(q32) - m0) / m0,
                             "status": s.status() | s64.status(),
                             "roofline": roofline(stage_flops(N_CELLS, ORDER, s.ghost_nnz()[0]),
                                                  3e3 / ms, fp32_peak)}
    del s64, s, q64, q32, q, qa
    # precision form, discontinuous flow: WENO9 dam break (2:1), C90, two days; FP64 with
    # epsilon 1e-40 and with 1e-12 (the FP32 epsilon: same scheme, arithmetic error alone)
    nd = 2 * day
    runs, nnz = {}, {}
    for name, P, eps in (("fp64", hp.HOPE_FP64, 1e-40), ("fp64_eps12", hp.HOPE_FP64, 1e-12),
                         ("fp32", hp.HOPE_FP32, 1e-12)):
        sw = hp.Sphere(N_CELLS, 9, hp.HOPE_WENO2D, P, omega=0.0, weno_eps=eps)
        nnz[name] = sw.ghost_nnz()[0]
        qw = sw.dam_break(h_in=10.0, h_out=5.0)
        m0 = sw.mass(qw)
        warm = qw.clone()
        with torch.cuda.stream(stream):
            sw.step(warm, 300.0, 1)
        ms_run = _run(sw, qw, 300.0, day, stream)
        h_day1 = qw[0].double().clone()
        ms_run += _run(sw, qw, 300.0, nd - day, stream)
        runs[name] = (qw, ms_run / nd, (sw.mass(qw) - m0) / m0, sw.status(), h_day1)
        del sw
    d1 = {name: runs[name][4] for name in runs}
    h64, h64b, h32 = runs["fp64"][0][0], runs["fp64_eps12"][0][0], runs["fp32"][0][0]
    for name in ("fp64", "fp32"):
        qw, msr, drift, st, _ = runs[name]
        out["weno9_c90_dam_" + name] = {"value": cells * 3 / (msr * 1e-3), "ms_per_step": msr,
                                        "days": nd * 300.0 / 86400.0, "mass_drift": drift, "status": st,
                                        "roofline": roofline(stage_flops(N_CELLS, 9, nnz[name], weno=True),
                                                             3e3 / msr,
                                                             fp64_peak if name == "fp64" else fp32_peak)}
    out["weno9_c90_dam_fp32"].update({"rel_l2_h_vs_fp64": _rel(h32, h64),
                                      "rel_l2_h_vs_fp64_same_eps": _rel(h32, h64b),
                                      "rel_l2_h_fp64_eps_1e-12_vs_1e-40": _rel(h64b, h64),
                                      # day 1: the configured epsilon pair (1e-12 in FP32, 1e-40 in
                                      # FP64) and the same-epsilon (arithmetic only) figure
                                      "day1_rel_l2_h_vs_fp64_eps_1e-12_vs_1e-40": _rel(d1["fp32"], d1["fp64"]),
                                      "day1_rel_l2_h_vs_fp64_same_eps": _rel(d1["fp32"], d1["fp64_eps12"]),
                                      "day1_bound": 1e-5})
    del runs, h64, h64b, h32
    # differentiation form: C180 WENO5, geostrophic + 16 bumps of 50 m, 50 steps of 150 s
    # with recompute from checkpoints every 10 steps; loss 0.5 |h_T - h_target|^2
    cen, cen_t = bump_centres(16, 0), bump_centres(16, 1)
    nsteps, every = 50, 10
    grads = {}
    for name, P in (("adjoint_c180_weno5_fp64", hp.HOPE_FP64), ("adjoint_c180_weno5_fp32", hp.HOPE_FP32)):
        s = hp.Sphere(180, 5, hp.HOPE_WENO2D, P)
        q0 = s.bumps(cen)
        target = s.bumps(cen_t)[0].clone()
        times = []
        with torch.cuda.stream(stream):
            for rep in range(2):  # the first pass captures the step graphs
                e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                x = q0.clone().requires_grad_(True)
                torch.cuda.synchronize()
                e[0].record(stream)
                qT = s.rollout(x, 150.0, nsteps, checkpoint_every=every)
                e[1].record(stream)
                loss = 0.5 * ((qT[0] - target) ** 2).sum()
                loss.backward()
                e[2].record(stream)
                torch.cuda.synchronize()
                times.append((e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])))
        fwd, bwd = times[-1]
        grads[name] = x.grad.double()
        c180 = 6 * 180 * 180 * 3 * nsteps
        fl = stage_flops(180, 5, s.ghost_nnz()[0], weno=True)
        pk = fp64_peak if P == hp.HOPE_FP64 else fp32_peak
        # forward + adjoint: the forward run, the backward's recompute of every step from
        # its checkpoint, and the reverse stages, an adjoint stage counted as twice the
        # forward stage's algorithmic FLOPs (the transposed linear maps cost the forward's
        # multiply-adds, the nonlinear weights' derivatives one more pass of that size)
        fa_flops = fl * 3 * nsteps * (1 + 1 + 2)
        out[name] = {"forward": c180 / (fwd * 1e-3), "forward_plus_adjoint": c180 / ((fwd + bwd) * 1e-3),
                     "steps": nsteps, "checkpoint_every": every, "fwd_ms": fwd, "adjoint_ms": bwd,
                     "adjoint_over_forward": bwd / fwd, "status": s.status(),
                     "roofline_forward": roofline(fl, 3 * nsteps / (fwd * 1e-3), pk),
                     "roofline_forward_plus_adjoint": {
                         "bound": "alu", "flops": fa_flops, "achieved_tflops": fa_flops / ((fwd + bwd) * 1e-3) / 1e12,
                         "peak_tflops": pk / 1e12, "frac": fa_flops / ((fwd + bwd) * 1e-3) / pk,
                         "convention": "forward run + recompute + reverse stages at 2x the forward stage FLOPs"}}
        del s
    out["adjoint_c180_weno5_fp32"]["rel_l2_grad_vs_fp64"] = _rel(grads["adjoint_c180_weno5_fp32"],
                                                                 grads["adjoint_c180_weno5_fp64"])
    del grads
    # batching form: 64 members (32 x C48, 24 x C96, 8 x C192), TPP7, FP32, RH + 1% noise;
    # one simulated day of 45 s steps, then the adjoint of the last 20 steps
    members, ens, q = ensemble_members(hp, hp.HOPE_FP32)
    dte, nday, nadj = 45.0, int(round(86400.0 / 45.0)), 20
    m0 = ens.mass(q)
    warm = q.clone()
    ms = _time_steps(ens, warm, dte, 20, stream)
    day_ms = _run(ens, q, dte, nday - nadj, stream)
    total = sum(6 * n * n for n in members)
    with torch.cuda.stream(stream):
        target = q[:].clone()
        # warm-up of the reverse sweep (adjoint scratch, member tables, tapes, step graphs of
        # the recompute buffers): one-time set-up, not part of the timed adjoint
        xw = q.clone().requires_grad_(True)
        (ens.rollout(xw, dte, 2, checkpoint_every=2) - target).square().sum().backward()
        del xw
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        x = q.clone().requires_grad_(True)
        torch.cuda.synchronize()
        e[0].record(stream)
        qT = ens.rollout(x, dte, nadj, checkpoint_every=10)
        e[1].record(stream)
        loss = 0.5 * ((qT - target) ** 2).sum()
        loss.backward()
        e[2].record(stream)
        torch.cuda.synchronize()
    fwd20, adj20 = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    m1 = ens.mass(qT.detach())
    ens_stage_flops = sum(stage_flops(n, 7, 0) for n in members) + 10 * ens.ghost_nnz()[0]
    fa_flops = ens_stage_flops * 3 * nadj * (1 + 1 + 2)  # as for the differentiation form
    out["ensemble64_tpp7_fp32"] = {"value": total * 3 / (ms * 1e-3), "ms_per_step": ms, "cells": total,
                                   "launches_per_stage": ens.launches_per_stage(),
                                   "day_s": (day_ms + fwd20) * 1e-3, "steps": nday,
                                   "day_value": total * 3 * nday / ((day_ms + fwd20) * 1e-3),
                                   "adjoint_steps": nadj, "adjoint_ms": adj20,
                                   "forward_plus_adjoint": total * 3 * nadj / ((fwd20 + adj20) * 1e-3),
                                   "max_member_mass_drift": max(abs(b - a) / a for a, b in zip(m0, m1)),
                                   "status": ens.status(),
                                   "roofline": roofline(ens_stage_flops, 3e3 / ms, fp32_peak),
                                   "roofline_forward_plus_adjoint": {
                                       "bound": "alu", "flops": fa_flops,
                                       "achieved_tflops": fa_flops / ((fwd20 + adj20) * 1e-3) / 1e12,
                                       "peak_tflops": fp32_peak / 1e12,
                                       "frac": fa_flops / ((fwd20 + adj20) * 1e-3) / fp32_peak,
                                       "convention": "forward run + recompute + reverse stages at 2x the forward "
                                                     "stage FLOPs"}}
    del ens, q, qT, x, warm, target
    # section 5.5: genuine-2D WENO-Z against the dimension-by-dimension comparator on the
    # C90 dam break (isotropy of the front), each with its throughput and roofline fraction
    try:
        out["dam_anisotropy_c90_weno5"] = anisotropy_form(hp, stream, fp64_peak)
    except Exception as exc:  # noqa: BLE001
        out["dam_anisotropy_c90_weno5"] = {"error": repr(exc)}
    # section 5.4: the perturbed jet as a second workload
    try:
        out["jet_c90_fp64"] = jet_form(hp, stream, fp64_peak)
    except Exception as exc:  # noqa: BLE001
        out["jet_c90_fp64"] = {"error": repr(exc)}
    # bottom topography: section 5.2's mountain flow against the flat step (the form is
    # reported, not the headline; a failure here is recorded instead of ending the run)
    try:
        out["mountain_c90_tpp11_fp64"] = mountain_form(hp, 96)
    except Exception as exc:  # noqa: BLE001
        out["mountain_c90_tpp11_fp64"] = {"error": repr(exc)}
    return out


def cpu_baseline(stages):
    """The FP64 C oracle (test infrastructure), as it stands, on this host's cores:
    `stages` tendency evaluations of the full workload."""
    from oracle import oracle as O
    o = O.Oracle(N_CELLS, ORDER, coriolis_tilt=ALPHA)
    q = o.geostrophic(ALPHA)
    o.tendency(q)  # warm-up (thread pool)
    t0 = time.perf_counter()
    for _ in range(stages):
        o.tendency(q)
    dt = time.perf_counter() - t0
    return 6 * N_CELLS * N_CELLS * stages / dt, dt


def run_reference(args, world, rank):
    if rank != 0:
        return
    from oracle import oracle as O
    o = O.Oracle(N_CELLS, ORDER, coriolis_tilt=ALPHA)
    q = o.geostrophic(ALPHA)
    for _ in range(max(args.warmup, 1)):
        o.tendency(q)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.tendency(q)
    el = time.perf_counter() - t0
    v = 6 * N_CELLS * N_CELLS * args.steps / el
    cores = os.cpu_count()
    sample = ("each step is one stage (one tendency evaluation) of the full workload, %d steps, "
              "C FP64 oracle with OpenMP over %d host threads" % (args.steps, cores))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "cell-stage/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (analytic steady geostrophic flow)",
            "config": {"workload": WORKLOAD, "N": N_CELLS, "order": ORDER, "scheme": "TPP"},
            "cpu_baseline": {"value": v, "unit": "cell-stage/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "cell-stage/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def ensemble_members(hp, precision, members=None):
    """The batching-form ensemble: 32 x C48, 24 x C96, 8 x C192 (or `members`), TPP7,
    Rossby-Haurwitz wave 4 with seeded 1 % h noise per member."""
    import torch
    from synth import noise_field
    if members is None:
        members = [48] * 32 + [96] * 24 + [192] * 8
    ens = hp.Sphere(members, 7, hp.HOPE_TPP, precision)
    q = ens.empty()
    for N in sorted(set(members)):
        base = hp.Sphere(N, 7, hp.HOPE_TPP, precision).rossby_haurwitz()
        for m, Nm in enumerate(members):
            if Nm == N:
                xi = torch.from_numpy(noise_field((6, N, N), 0, member=m)).to("cuda", base.dtype)
                ens.member(q, m).copy_(base * (1 + 0.01 * xi)[None])
    return members, ens, q


def mountain_form(hp, steps):
    """Section 5.2's flow over the isolated mountain (eq. 5.8) at C90, TPP11, FP64, SSP-RK3
    dt = 150 s (300 s is unstable for this unlimited scheme on the cone's kinks at C90),
    against the same graph-replayed step of the flat steady flow (h0 = 5960 m, u0 = 20 m/s)
    without a surface; `steps` timed steps of each."""
    import torch
    s = hp.Sphere(90, 11)
    dt = 150.0
    cases = (("flat", None, s.geostrophic(0.0, 20.0, 5960.0 * s.gravity)),
             ("mountain", s.mountain_surface(), s.mountain_flow()))
    out = {"steps": steps, "dt_s": dt}
    for label, topo, q0 in cases:
        s.set_topography(topo)
        q = q0.clone()
        s.step(q, dt, 3)
        q.copy_(q0)
        m0 = s.mass(q)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        e[0].record()
        s.step(q, dt, steps)
        e[1].record()
        torch.cuda.synchronize()
        ms = e[0].elapsed_time(e[1])
        out[label] = {"ms_per_step": ms / steps,
                      "cell_stage_per_s": 3 * 6 * 90 * 90 * steps / (ms * 1e-3),
                      "mass_drift": abs(s.mass(q) - m0) / abs(m0),
                      "launches_per_stage": s.launches_per_stage(), "status": s.status()}
    out["mountain_over_flat_time"] = out["mountain"]["ms_per_step"] / out["flat"]["ms_per_step"]
    return out


def anisotropy_form(hp, stream, fp64_peak, days=2.0, N=90):
    """Section 5.5's comparison: the cylinder dam break (10 m inside a 20-degree cap at
    (0, 0), 5 m outside, at rest, Omega = 0; the 2:1 ratio of eq. 5.19) at C90, fifth order,
    FP64, SSP-RK3 dt = 300 s, with the genuine-2D WENO-Z, the dimension-by-dimension
    comparator and the unlimited TPP5 as a linear reference.  After each simulated day the
    azimuthal spread of h about the dam centre and the grid-axis / diagonal difference of
    its residual profile (front_anisotropy) are recorded, with each run's throughput and
    roofline fraction."""
    import torch
    dt = 300.0
    nday = int(round(86400.0 / dt))
    lon, lat, sg = cell_geometry(N)
    dcell = np.pi / (2 * N)
    out = {"N": N, "order": 5, "dt_s": dt, "days": days, "h_in_m": 10.0, "h_out_m": 5.0,
           "cap_deg": 20.0, "fp64_peak_tflops": fp64_peak / 1e12}
    for name, scheme, wflag in (("weno2d", hp.HOPE_WENO2D, True), ("weno1d", hp.HOPE_WENO1D, "1d"),
                                ("tpp5", hp.HOPE_TPP, False)):
        s = hp.Sphere(N, 5, scheme, hp.HOPE_FP64, omega=0.0)
        q0 = s.dam_break(h_in=10.0, h_out=5.0)
        q = q0.clone()
        m0 = s.mass(q)
        with torch.cuda.stream(stream):
            s.step(q, dt, 2)  # captures this buffer's step graph (FP64: no low word to reset)
        torch.cuda.synchronize()
        q.copy_(q0)
        res, ms_tot = {}, 0.0
        for d in range(int(round(days))):
            ms_tot += _run(s, q, dt, nday, stream)
            h = (q[0].double().cpu().numpy() / sg) / s.gravity
            res["day%d" % (d + 1)] = front_anisotropy(h, lon, lat, 0.0, 0.0, dcell, 5.0, np.radians(60.0))
        msr = ms_tot / (nday * int(round(days)))
        fl = stage_flops(N, 5, s.ghost_nnz()[0], weno=wflag)
        res.update({"value": 6 * N * N * 3 / (msr * 1e-3), "ms_per_step": msr,
                    "mass_drift": (s.mass(q) - m0) / m0, "status": s.status(),
                    "roofline": roofline(fl, 3e3 / msr, fp64_peak)})
        out[name] = res
        del s, q, q0
    return out


def jet_form(hp, stream, fp64_peak, hours=24.0, N=90):
    """Section 5.4's perturbed jet (eqs. 5.16-5.18) as a second workload at C90, FP64, with
    the headline's TPP11 and with WENO5, SSP-RK3 dt = 150 s (the jet's 80 m/s plus the
    gravity-wave speed put 300 s near the stability limit at this resolution); throughput,
    roofline fraction and mass drift over `hours` simulated hours."""
    import torch
    dt = 150.0
    n = int(round(hours * 3600.0 / dt))
    out = {"N": N, "dt_s": dt, "hours": hours, "steps": n}
    for name, scheme, k, wflag in (("tpp11", hp.HOPE_TPP, 11, False), ("weno5", hp.HOPE_WENO2D, 5, True)):
        s = hp.Sphere(N, k, scheme, hp.HOPE_FP64)
        q0 = s.galewsky()
        q = q0.clone()
        m0 = s.mass(q)
        with torch.cuda.stream(stream):
            s.step(q, dt, 2)
        torch.cuda.synchronize()
        q.copy_(q0)
        ms = _run(s, q, dt, n, stream) / n
        fl = stage_flops(N, k, s.ghost_nnz()[0], weno=wflag)
        out[name] = {"value": 6 * N * N * 3 / (ms * 1e-3), "ms_per_step": ms,
                     "mass_drift": (s.mass(q) - m0) / m0, "status": s.status(),
                     "finite": bool(torch.isfinite(q).all().item()),
                     "roofline": roofline(fl, 3e3 / ms, fp64_peak)}
        del s, q, q0
    return out


def run_case(args):
    """Short single-form runs for profiling (`--case`): not the benchmark line."""
    import torch
    import paper_2411_19185_gb300 as hp
    if args.case == "ensemble64":
        members, ens, q = ensemble_members(hp, hp.HOPE_FP32)
        ens.step(q, 45.0, 3)
        ens.set_profiling(True)
        ens.step(q, 45.0)
        acc = np.zeros(4)
        for _ in range(10):
            ens.step(q, 45.0)
            acc += np.sum(np.array(ens.kernel_times()), axis=0)
        ens.set_profiling(False)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "phase_ms_per_stage": dict(zip(["ghost", "recon", "flux", "update"],
                                                                        (acc / 30).tolist())),
                          "status": ens.status()}))
        return
    if args.case == "mountain_c90_tpp11_fp64":
        print(json.dumps({"case": args.case, **mountain_form(hp, args.steps)}))
        return
    if args.case == "weno1d_c90":
        # the comparator's stage at C90 (dam break, FP64), a few graph-replayed steps
        s = hp.Sphere(90, 5, hp.HOPE_WENO1D, hp.HOPE_FP64, omega=0.0)
        q = s.dam_break(h_in=10.0, h_out=5.0)
        s.step(q, 300.0, args.steps)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "steps": args.steps, "status": s.status()}))
        return
    if args.case in ("ensemble64_adjoint", "ensemble16_adjoint"):
        # the batching form's reverse sweep: a taped rollout of args.steps steps and its
        # backward (persistent forward and VJP launches); ensemble16: 8 x C96 + 8 x C48, a
        # case small enough for a full profiler capture
        small = [96] * 8 + [48] * 8 if args.case == "ensemble16_adjoint" else None
        members, ens, q = ensemble_members(hp, hp.HOPE_FP32, small)
        x = q.clone().requires_grad_(True)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        qT = ens.rollout(x, 45.0, args.steps, checkpoint_every=args.steps)
        e[1].record()
        (qT * qT).sum().backward()
        e[2].record()
        torch.cuda.synchronize()
        # phases of one taped reverse stage (profiling stamps at the VJP launch's barriers)
        tape = torch.empty(ens.tape_bytes(), dtype=torch.uint8, device="cuda")
        qr = q.clone()
        ens.step_record(qr, 45.0, tape)
        ens.set_profiling(True)
        ens.step_vjp_tape(q, tape, qr, 45.0)
        ph = ens.vjp_phase_times()
        ens.set_profiling(False)
        print(json.dumps({"case": args.case, "steps": args.steps, "fwd_ms": e[0].elapsed_time(e[1]),
                          "adjoint_ms": e[1].elapsed_time(e[2]), "status": ens.status(),
                          "last_reverse_stage_phase_ms": dict(zip(("fwd_ghost", "fwd_recon", "flux_adj",
                                                                   "recon_adj", "gather", "ghost_adj"), ph))}))
        return
    if args.case == "dam_anisotropy_c90":
        peak = hp.measure_fma_peak(hp.HOPE_FP64)
        print(json.dumps({"case": args.case, **anisotropy_form(hp, torch.cuda.current_stream(), peak)}))
        return
    from synth import bump_centres
    P = hp.HOPE_FP32 if args.case.endswith("fp32") else hp.HOPE_FP64
    s = hp.Sphere(180, 5, hp.HOPE_WENO2D, P)
    q0 = s.bumps(bump_centres(16, 0))
    target = s.bumps(bump_centres(16, 1))[0].clone()
    n = args.steps
    for rep in range(2):
        x = q0.clone().requires_grad_(True)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        e[0].record()
        qT = s.rollout(x, 150.0, n, checkpoint_every=10)
        e[1].record()
        loss = 0.5 * ((qT[0] - target) ** 2).sum()
        loss.backward()
        e[2].record()
        torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "steps": n, "fwd_ms": e[0].elapsed_time(e[1]),
                      "adjoint_ms": e[1].elapsed_time(e[2]), "status": s.status()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=288)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-stages", type=int, default=150)
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--case", choices=["ensemble64", "adjoint_c180_fp64", "adjoint_c180_fp32",
                                       "mountain_c90_tpp11_fp64", "dam_anisotropy_c90", "weno1d_c90",
                                       "ensemble64_adjoint", "ensemble16_adjoint"],
                    help="run one form briefly for profiling instead of the benchmark")
    args = ap.parse_args()
    if args.case:
        run_case(args)
        return
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2411_19185_gb300 as hp

    fp64_peak, peak_mhz, peak_fpc = hp.measure_fma_peak_clock(hp.HOPE_FP64, 8)
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    s = hp.Sphere(N_CELLS, ORDER, hp.HOPE_TPP, hp.HOPE_FP64, coriolis_tilt=ALPHA)
    q = s.geostrophic(ALPHA)
    q_analytic = q.clone()
    m0 = s.mass(q)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    cells = 6 * N_CELLS * N_CELLS
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            s.step(q, DT)
        s.set_profiling(True)
        s.step(q, DT)  # captures the profiled graph
        s.mass(q)
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        recon_ms = []
        kernel_sum = np.zeros(4)
        sampler = ClockSampler(local)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        sampler.start()
        for k in range(args.steps):
            flush.zero_()
            ev0[k].record(stream)
            s.step(q, DT)
            ev1[k].record(stream)
            s.mass(q)  # FP64 mass diagnostic, read back to the host (outside the timed events)
            kt = s.kernel_times()
            recon_ms.extend(st[1] for st in kt)
            kernel_sum += np.sum(np.array(kt), axis=0)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clocks = sampler.stop()
        total_ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
        s.set_profiling(False)
        # end to end through the C ABI with host buffers (copies inside the call)
        qh = q.detach().to("cpu").pin_memory()
        s.step_host(qh, DT, 1, out=qh)
        e2e_s = 0.0
        for k in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.step_host(qh, DT, 1, out=qh)
            e2e_s += time.perf_counter() - t0
    m1 = s.mass(q)
    status = s.status()
    # the workload is a steady state: the state after the run is compared with the analytic
    # cell averages it started from (steps taken: warm-up + profiled capture + timed)
    steps_run = args.warmup + 1 + args.steps
    err_h = float(torch.linalg.norm(q[0] - q_analytic[0]) / torch.linalg.norm(q_analytic[0]))
    forms = None
    if not args.no_forms:
        fs = ClockSampler(local)
        fs.start()
        forms = measure_forms(hp, stream, fp64_peak)
        forms["clocks"] = fs.stop()  # sampled over all form runs
    total_ms = reduce_max(total_ms, world)
    e2e_s = reduce_max(e2e_s, world)
    value = job_value(world, cells, args.steps, total_ms * 1e-3)
    e2e_value = job_value(world, cells, args.steps, e2e_s)
    recon_avg_ms = float(np.mean(recon_ms))
    flops = recon_flops_per_launch(N_CELLS, ORDER)
    flops_ev = recon_flops_evaluated_per_launch(N_CELLS, ORDER)
    achieved = flops / (recon_avg_ms * 1e-3)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "cell-stage/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (analytic steady geostrophic flow, eqs. 5.1-5.3)",
        "config": {"workload": WORKLOAD, "N": N_CELLS, "order": ORDER, "scheme": "TPP", "dt_s": DT,
                   "l2": "flushed before every timed step (512 MiB write); state 1.2 MB is L2-resident",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"kernel": "k_recon_tpp<double,11>", "bound": "alu", "achieved": achieved / 1e12,
                     "peak": fp64_peak / 1e12, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                     "peak_source": "FP64 FMA microbenchmark measured in this run (hope_measure_fma_peak_clock)",
                     "peak_sm_mhz": peak_mhz, "peak_flops_per_sm_clock": peak_fpc,
                     "flops_per_launch": flops, "avg_launch_ms": recon_avg_ms,
                     "traffic": RECON_TRAFFIC_BYTES if RECON_TRAFFIC_CURRENT else None,
                     "traffic_last_capture": RECON_TRAFFIC_BYTES,
                     # the same outputs as the kernel evaluates them (mirror pairs): fewer
                     # operations, so the measurement plan's count above reads above the
                     # FMA peak while the FP64 pipe itself is about 80 % busy
                     "flops_per_launch_evaluated": flops_ev,
                     "frac_evaluated": flops_ev / (recon_avg_ms * 1e-3) / fp64_peak},
        "stage_kernel_ms": {"ghost": kernel_sum[0] / (3 * args.steps), "recon": kernel_sum[1] / (3 * args.steps),
                            "flux": kernel_sum[2] / (3 * args.steps), "update": kernel_sum[3] / (3 * args.steps)},
        "e2e": {"value": e2e_value, "unit": "cell-stage/s", "h2d_bytes_per_step": q.numel() * 8,
                "d2h_bytes_per_step": q.numel() * 8},
        "gpu_launches": args.steps * (3 * s.launches_per_stage() + 2),
        "clocks": clocks,
        "mass_drift": (m1 - m0) / m0,
        "error_vs_analytic": {"rel_l2_sqrtG_phi": err_h, "steps": steps_run,
                              "days": steps_run * DT / 86400.0},
        "device_status": status,
        "forms": forms,
    }
    # the same fraction with the peak taken at the clock sampled during the timed region:
    # the microbenchmark's flops per SM per cycle x SMs x median SM MHz of the run
    if clocks and clocks.get("sm_mhz"):
        peak_run = peak_fpc * nsm * clocks["sm_mhz"] * 1e6
        line["roofline"]["peak_at_run_clock"] = peak_run / 1e12
        line["roofline"]["frac_at_run_clock"] = achieved / peak_run
    g_nnz = s.ghost_nnz()[0]
    hbm_bps, hbm_src = measured_hbm_bps()
    line["step_roofline"] = step_roofline(stage_flops(N_CELLS, ORDER, g_nnz), 72 * cells, 12 * g_nnz,
                                          total_ms * 1e-3 / args.steps / 3, fp64_peak, hbm_bps)
    line["step_roofline"]["hbm_source"] = hbm_src
    fl_ev = stage_flops(N_CELLS, ORDER, g_nnz, evaluated=True)
    line["step_roofline"]["evaluated"] = {
        "flops_per_stage": fl_ev, "frac": fl_ev / fp64_peak / (total_ms * 1e-3 / args.steps / 3)}
    if forms:
        for name, f in forms.items():
            if isinstance(f, dict) and ("value" in f or "forward" in f):
                f["vs_fp64_path"] = f.get("value", f.get("forward")) / value
    if world == 1 and not args.no_cpu_baseline:
        v, el = cpu_baseline(args.cpu_stages)
        line["cpu_baseline"] = {"value": v, "unit": "cell-stage/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": "%d tendency evaluations (stages) of the full workload, %.1f s" %
                                          (args.cpu_stages, el),
                                "cpu_model": cpu_model()}
        if set_host_threads(1):
            v1, el1 = cpu_baseline(max(1, args.cpu_stages // 30))
            set_host_threads(os.cpu_count())
            line["cpu_baseline"]["single_core"] = {"value": v1, "sample": "%d stages, %.1f s" %
                                                   (max(1, args.cpu_stages // 30), el1)}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
