#!/usr/bin/env python
"""Benchmark of the per-pixel ray integration path.

Workload: the twisted bar (single cubic B-spline block, 8x8x32 control points,
parametrisation-quality scalar, Eq. 23) rendered at 1920x1080 with a
perspective camera, plain FP32, RK tolerance 1e-5, ds = diag/128, K = 4.
One step = one whole frame: face projection, ray/face intersection,
depth sort + Alg. 2 pairing, and ODE integration with compositing.

Prints one JSON line.  `value` is Mpixels/s over the whole job (all ranks),
timed on the device with CUDA events per step; L2 is flushed (a 512 MiB
write) between timed steps, outside the events.  `e2e` is the same metric
through ivv_render_to_host (pinned host output, device->host copy inside).
`--impl reference` times the FP64 CPU oracle on a bounded row sample.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixels/s & ms/frame at 1920x1080 vs plain FP32, at <=1e-3 max RGBA error"
UNIT = "Mpixels/s"
WORKLOAD = "twisted bar, 1 cubic block 8x8x32 cp, quality scalar (Eq. 23), 1920x1080 perspective, FP32"

RK_NAMES = {1: "Euler (RK1)", 2: "midpoint (RK2)", 3: "Kutta-3 (RK3)", 4: "RK4", 5: "RK4 3/8", 6: "Fehlberg-5 (RKF)",
            7: "implicit Euler (IRK1)"}

# --workload: the default is the headline frame above; the others are the
# remaining workloads of the method, each printed as its own line.
WORKLOADS = {
    "bar1080": (1, 0, WORKLOAD),
    "cube64-fp64": (0, 2, "twisted cube, 1 cubic Bezier element, 64x64 orthographic, rk_tol 1e-8, FP64"),
    "beam1080": (2, 1, "bent beam, 16 cubic blocks 6x6x12 cp (C0), Gaussian-sum scalar, 1920x1080 perspective, "
                       "mixed precision"),
    "beam1080-fp32": (2, 0, "bent beam, 16 cubic blocks 6x6x12 cp (C0), Gaussian-sum scalar, 1920x1080 "
                            "perspective, FP32"),
    "backstep4k": (4, 1, "backward-facing step, 3 quadratic/cubic blocks 64x16x16 cp, shear-layer scalar, "
                         "64-knot TF, 3840x2160, rk_tol 7e-7, mixed precision"),
    "backstep4k-fp32": (4, 0, "backward-facing step, 3 quadratic/cubic blocks 64x16x16 cp, shear-layer scalar, "
                              "64-knot TF, 3840x2160, rk_tol 7e-7, FP32"),
    "beam1080-vonmises": ("vm", 0, "bent beam, 16 cubic blocks 6x6x12 cp (C0) with a cantilever displacement "
                                   "spline, von Mises scalar (6.2, Eq. 24), 1920x1080 perspective, FP32"),
    "batch64": (None, 0, "64 requests over the twisted cube, twisted bar and bent beam, sizes uniform over "
                         "{256,512,768,1024}^2, seeded cameras and TFs, FP32, one CUDA graph"),
}

# Workloads of the learned initial guess: (base workload, render-parameter
# overrides, label).  The guess network (3-64-64-3 per block) is trained on
# the device before the timed frames (2^20 forward-map samples per block,
# untimed, reported as train_s).  RF: every sample's Newton starts from the
# guess named; rf_tol 1e-3 of the pixel half width (image parity, not only
# pixel accuracy).
LEARNED_WORKLOADS = {
    "beam1080-rf-learned-mixed": ("beam1080", {"method": 1, "use_mlp_guess": 1, "rf_tol": 1e-3},
                                  "root finding per sample (5.1) from the learned guess, mixed precision"),
    "beam1080-rf-chord-fp32": ("beam1080-fp32", {"method": 1, "use_mlp_guess": 2, "rf_tol": 1e-3},
                               "root finding per sample (5.1) from the chord guess, FP32"),
    "bar1080-rf-learned-mixed": ("bar1080", {"precision": 1, "method": 1, "use_mlp_guess": 1, "rf_tol": 1e-3},
                                 "root finding per sample (5.1) from the learned guess, mixed precision"),
    "bar1080-rf-chord-fp32": ("bar1080", {"method": 1, "use_mlp_guess": 2, "rf_tol": 1e-3},
                              "root finding per sample (5.1) from the chord guess, FP32"),
    "backstep4k-rf-learned-mixed": ("backstep4k", {"method": 1, "use_mlp_guess": 1, "rf_tol": 1e-3},
                                    "root finding per sample (5.1) from the learned guess, mixed precision"),
    "backstep4k-rf-chord-fp32": ("backstep4k-fp32", {"method": 1, "use_mlp_guess": 2, "rf_tol": 1e-3},
                                 "root finding per sample (5.1) from the chord guess, FP32"),
    "beam1080-learned-mixed": ("beam1080", {"use_mlp_guess": 1},
                               "ODE method with the learned guess for stage-2 entries without chord context "
                               "(none on this view: the guess network is idle)"),
}


def kernels_per_frame(prec, rk_method, method=0, guess=0, n_blocks=1):
    """Kernels one frame of the benchmark's workloads launches: stages 1-2
    (K0, K2a, K2b, both K2c forms, K4, which also counts the sample lists;
    mixed precision adds the K2p polish of grazing hits) and stage 3 -- the
    split integration (K5t, shading), one fused integrator (FP64, fixed-step,
    implicit Euler), or the RF chain (expansion, Newton, compositing, plus
    the guess network's inference with the learned guess, after a
    three-kernel block sort for volumes of 8 blocks or more).  Frames with
    cutting or near planes or singular faces count their samples with four
    more kernels after the fix-up solves; none of the workloads has them."""
    n = 6 + (1 if prec == 1 else 0)
    if method == 1:
        return n + 3 + ((1 + (3 if n_blocks >= 8 else 0)) if guess == 1 else 0)
    return n + (2 if prec != 2 and not rk_method else 1)


# A batch replays the same stages for every request at once, plus the
# overflow list and its fused integrator.
BATCH_KERNELS = 14


# Algorithmic FP32 flops per unit for Bezier degree P (N = P + 1 control
# points per direction; the cubic figures in brackets).
def flop_model(P):
    N = P + 1
    return {
        # one W(p): sum-factorised phi + J (6N^3 + 9N^2 + 12N FMA [576]), Bernstein
        # basis, V and the 3x3 adjugate solve (131) [1283]
        "rhs": 2 * (6 * N ** 3 + 9 * N ** 2 + 12 * N) + 131,
        # stage combinations, clamps and error norm of one BS3(2) step attempt [70]
        "step": 70,
        # K=4 supersampled TF lookups + Alg. 1 updates per sample [150]
        "sample": 150,
        # scalar at a sample evaluated on its own (shading pass of the split
        # integration): det J or Eq. 23 from J alone (6N^3 + 9N^2 + 9N FMA [564]),
        # basis, det and Frobenius norm [1220]; or the scalar control points
        # (N^3 + N^2 + N FMA [84]) and the value basis [200]
        "rho_j": 2 * (6 * N ** 3 + 9 * N ** 2 + 9 * N) + 92,
        "rho_cp": 2 * (N ** 3 + N ** 2 + N) + 32,
        # von Mises (§6.2): J_phi and J_u at the sample (two contractions of
        # 6N^3 + 9N^2 + 9N FMA, one basis), the adjugate, J_u adj(J) / det,
        # the strain's deviatoric sum and its root (130) [2348]
        "rho_vm": 4 * (6 * N ** 3 + 9 * N ** 2 + 9 * N) + 92 + 130,
        # one implicit Euler Newton iteration: phi, J and the Hessian
        # (9N^3 + 18N^2 + 30N FMA [984]), second-derivative basis, V and the
        # solve for W, the Jacobian of G and its solve [2218]
        "irk": 2 * (9 * N ** 3 + 18 * N ** 2 + 30 * N) + 250,
        # ray/patch intersection (K2): per (pixel, patch) item the N^2 control
        # points into the ray frame (6 FMA each), hull and Jacobian-sign test [260];
        # one 2-D Newton iteration (value, 2 partials: 4N^2 + 6N FMA, 2x2 solve) [230];
        # per fragment the 3-D point, partials and facing [220]
        "hull": 12 * N * N + 68,
        "newton": 2 * (4 * N * N + 6 * N) + 54,
        "frag": round(220 * (6 * N * N + 9 * N) / 132),
    }


def scene_degree(blocks):
    """The common Bezier degree the library raises a volume's blocks to."""
    return max(max(b.degree) for b in blocks)


def _scalar_kind(mode):
    return {0: "cp", 3: "vm"}.get(int(mode), "j")


def k5_flops_per_unit(st, F, scalar_mode, P):
    """Stage-3 work of the frame priced per unit with the scalar taken as if
    J were at hand at every sample: per RHS F["rhs"] (1283 cubic), per step
    attempt 40, per sample 100 (K = 4 TF lookups, exp and Alg. 1) plus the
    scalar, N^3 + N^2 + N FMA from control points or about 40 flop from J
    (det J, Eq. 23).  The shading pass of the split integration pays a fresh
    J at each sample instead (rho_evals x F["rho_j"]): that cost of the
    split design is not counted here."""
    N = P + 1
    kind = _scalar_kind(scalar_mode)
    # the scalar with J at hand: control points; det J or Eq. 23 (about 40);
    # von Mises: the J_u contraction (6N^3 + 9N^2 + 9N FMA) and 130
    rho = {"cp": 2 * (N ** 3 + N ** 2 + N), "j": 40, "vm": 2 * (6 * N ** 3 + 9 * N ** 2 + 9 * N) + 130}[kind]
    return st["rhs_evals"] * F["rhs"] + (st["rk_steps"] + st["rk_rejects"]) * 40 + st["samples"] * (100 + rho)


def k5_flops(st, F, scalar_mode, implicit=False):
    # implicit Euler counts one map evaluation per Newton iteration in rhs_evals
    return (st["rhs_evals"] * (F["irk"] if implicit else F["rhs"])
            + (st["rk_steps"] + st["rk_rejects"]) * F["step"]
            + st["samples"] * F["sample"] + st["rho_evals"] * F["rho_" + _scalar_kind(scalar_mode)])


def k2_flops(st, F):
    return st["isect_items"] * F["hull"] + st["isect_newton"] * F["newton"] + st["fragments"] * F["frag"]


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm_sorted = sorted(sm)
        return {"sm_mhz": sm_sorted[len(sm_sorted) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _gpu_id_for_smi(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return local_rank


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def _ncu_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` from the committed ncu counters, or
    None if they were taken on another workload or its sources changed since
    the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_counters.json")) as f:
            rec = json.load(f)[kernel]
        if rec.get("workload") != workload:
            return None
        m = hashlib.sha256()
        for name in rec["src_files"]:
            with open(os.path.join(ROOT, "paper_1404_3363_gb300", "csrc", name), "rb") as f:
                m.update(f.read())
        return rec["dram_bytes_per_launch"] if m.hexdigest()[:16] == rec["src_sha"] else None
    except (OSError, KeyError, ValueError):
        return None


def cpu_oracle_sample(scene, target_s=12.0, max_stride=64, label="1920x1080 frame"):
    """Oracle Mpix/s on evenly spaced rows of the frame (rows at stride s,
    halving s until one sample takes >= target_s / 3).  Returns the
    cpu_baseline record and the rendered rows {y: float64 [W][4]}."""
    import oracle
    vol = oracle.OracleVolume(scene.blocks, scene.scalar_mode)
    W, H = scene.width, scene.height
    stride = max_stride
    best = None
    cores = os.cpu_count() or 1
    while True:
        rows = list(range(stride // 2, H, stride))
        got = {}
        t0 = time.perf_counter()
        for y in rows:
            got[y] = oracle.render(scene, vol, window=(0, W, y, y + 1), n_threads=cores)[0]
        dt = time.perf_counter() - t0
        best = (len(rows) * W, dt, stride, len(rows), got)
        if dt >= target_s / 3 or stride == 1:
            break
        stride //= 2
    px, dt, stride, nrows, got = best
    return {"value": px / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d rows at stride %d of the %s (%d pixels), FP64 per-sample Newton, "
                      "%.2f s" % (nrows, stride, label, px, dt)}, got


def image_parity(img, rows):
    """Max |dRGBA| of the device image against the oracle's rows."""
    import numpy as np
    err = 0.0
    for y, ref in rows.items():
        err = max(err, float(np.abs(img[y].astype(np.float64) - ref).max()))
    return {"max_rgba_err": err, "pixels": len(rows) * img.shape[1], "rows": len(rows),
            "tolerance": 1e-3, "ok": err <= 1e-3}


def pair_parity(vol, sc, rows):
    """Entry/exit points (stage 1-2 result) of the frame's rows against the
    oracle's FP64 intersections: parameter-space error per image, over all
    hits and over the hits at least 0.2 away from grazing (|cos| of the ray
    and the face normal), and pixels whose pair count differs."""
    import numpy as np
    import oracle
    W, H = sc.width, sc.height
    cores = os.cpu_count() or 1
    ov = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    ys = sorted(rows)
    if len(ys) == H:
        co, po, bo = ov.window_pairs(sc.camera, W, H, n_threads=cores)
    else:
        parts = [ov.window_pairs(sc.camera, W, H, window=(0, W, y, y + 1), n_threads=cores) for y in ys]
        co = np.concatenate([q[0] for q in parts])
        po = np.concatenate([q[1] for q in parts], axis=1)
        bo = np.concatenate([q[2] for q in parts], axis=1)
    cap = max(1, int(co.max()))
    cg, pg, bg = vol.render_pairs(sc.camera, sc.params, W, H, max_pairs=cap)
    sel = (np.array(ys)[:, None] * W + np.arange(W)[None, :]).reshape(-1)
    cg = cg.cpu().numpy()[sel]
    pg = pg.cpu().numpy()[:, sel].astype(np.float64)
    bg = bg.cpu().numpy()[:, sel]
    same = cg == co
    worst, worst_ng, worst_t, n_hits, n_graze, blk_bad = 0.0, 0.0, 0.0, 0, 0, 0
    for k in range(cap):
        m = same & (co > k)
        if not m.any():
            continue
        blk_bad += int((bg[k][m] != bo[k][m]).sum())
        for a, b in ((0, 3), (4, 7)):
            got, ref = pg[k][m][:, a:b], po[k][m][:, a:b]
            e = np.abs(got - ref).max(axis=1)
            worst_t = max(worst_t, float(np.abs(pg[k][m][:, b] - po[k][m][:, b]).max()))
            cosg = np.ones(len(ref))
            for blk in np.unique(bo[k][m]):
                q = bo[k][m] == blk
                phi, J, _ = ov.eval(int(blk), ref[q])
                face = np.argmin(np.minimum(np.abs(ref[q]), np.abs(ref[q] - 1)), axis=1)
                nrm = np.linalg.inv(J)[np.arange(int(q.sum())), face]          # face normal: row of J^-1
                if sc.camera.ortho:
                    d = np.broadcast_to(np.asarray(sc.camera.target, float) - np.asarray(sc.camera.eye, float),
                                        phi.shape)
                else:
                    d = phi - np.asarray(sc.camera.eye, float)                 # the ray passes the eye
                cosg[q] = np.abs((nrm * d).sum(1)) / (np.linalg.norm(nrm, axis=1) * np.linalg.norm(d, axis=1))
            worst = max(worst, float(e.max()))
            ng = cosg >= 0.2
            if ng.any():
                worst_ng = max(worst_ng, float(e[ng].max()))
            n_hits += len(e)
            n_graze += int((~ng).sum())
    return {"pixels": int(len(sel)), "hits": n_hits, "grazing_hits": n_graze,
            "max_param_err": worst, "max_param_err_non_grazing": worst_ng, "max_t_err": worst_t,
            "count_mismatch_pixels": int((~same).sum()), "block_mismatch": blk_bad,
            "bound": 1e-5}


def tile_rows(height, rank, world):
    """Band of rows (y0, h) of a frame split over `world` ranks (--split
    rows): contiguous bands, the first height % world ranks one row taller."""
    base, extra = divmod(height, world)
    y0 = rank * base + min(rank, extra)
    return y0, base + (1 if rank < extra else 0)


def aggregate_ranks(ms_local, pixels_per_rank, dist=None, device=None):
    """Whole-job Mpixels/s: every rank renders its own frame (replicas, weak
    scaling); the job time is the slowest rank's.  Returns (value, ms_max)."""
    ms = float(ms_local)
    world = 1
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([ms], dtype=torch.float64, device=device or "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * pixels_per_rank / (ms * 1e-3) / 1e6, ms


def run_reference(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    from paper_1404_3363_gb300 import scenes
    import oracle
    sc = scenes.config(1)
    vol = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    W, H = sc.width, sc.height
    cores = os.cpu_count() or 1
    stride = args.ref_stride
    rows = list(range(stride // 2, H, stride))

    def step():
        for y in rows:
            oracle.render(sc, vol, window=(0, W, y, y + 1), n_threads=cores)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    px = len(rows) * W
    value = px / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "width": W, "height": H,
                   "sample": "%d rows at stride %d per step" % (len(rows), stride)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d rows at stride %d of the frame (%d pixels) per step" % (len(rows), stride, px)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_1404_3363_gb300 import build as libbuild
    libbuild.build()
    from paper_1404_3363_gb300 import ivv, scenes

    overrides, train = {}, False
    if args.workload in LEARNED_WORKLOADS:
        base, overrides, label = LEARNED_WORKLOADS[args.workload]
        cfg, prec, workload = WORKLOADS[base]
        workload = workload + ", " + label
        train = overrides.get("use_mlp_guess") == 1
    else:
        cfg, prec, workload = WORKLOADS[args.workload]
    sc = scenes.bent_beam(seed=12347, displacement=True) if cfg == "vm" else scenes.config(cfg)
    sc.params.precision = prec
    for k, v in overrides.items():
        setattr(sc.params, k, v)
    prec = sc.params.precision
    if args.rk_method:
        sc.params.rk_method = args.rk_method
        workload += ", fixed-step %s (one step per sample interval)" % RK_NAMES[args.rk_method]
    if args.c is not None:
        sc.params.c = args.c
        workload += ", c = %g" % args.c
    if args.rk_tol is not None:
        sc.params.rk_tol = args.rk_tol
        workload = workload.replace("rk_tol 7e-7", "rk_tol %g" % args.rk_tol)
        if "rk_tol" not in workload:
            workload += ", rk_tol %g" % args.rk_tol
    if train and (args.guess_samples != 1 << 20 or args.guess_epochs != 8):
        workload += ", guess trained on %d samples x %d epochs per block" % (args.guess_samples, args.guess_epochs)
    W, H = sc.width, sc.height
    FW, FH = W, H                     # the full frame
    window = None
    if args.split == "rows" and world > 1:
        # strong scaling: each rank renders its band of rows of the one frame
        y0, H = tile_rows(FH, rank, world)
        window = (0, y0, FW, FH)
    stream = torch.cuda.current_stream()
    vol = ivv.volume_for(sc)
    train_s = None
    if train:
        t0 = time.perf_counter()
        train_loss = vol.train_guess(samples_per_block=args.guess_samples, epochs=args.guess_epochs, batch=4096,
                                     lr=3e-3, seed=1)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    # untimed instrumented replay: algorithmic work counts of this exact frame
    vol.reset_stats()
    vol.render(sc.camera, sc.params, W, H, out=out, flags=ivv.FLAG_STATS, window=window)
    st = vol.stats()
    F = flop_model(scene_degree(sc.blocks))
    flops_k5 = k5_flops(st, F, sc.scalar_mode, implicit=args.rk_method == 7)
    flops_k5_unit = (k5_flops_per_unit(st, F, sc.scalar_mode, scene_degree(sc.blocks))
                     if args.rk_method != 7 and sc.params.method == 0 else None)
    flops_k2 = k2_flops(st, F)

    def frame(flags=0):
        vol.render(sc.camera, sc.params, W, H, out=out, flags=flags, window=window)

    for _ in range(args.warmup):
        frame()
        flush.zero_()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(_gpu_id_for_smi(local))
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        frame()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    # stage breakdown (and the roofline's stage times): the same frames again,
    # timed by the library's events between its stages.  Those records, and
    # reading them back after every frame, cost the frame about 3 %, so these
    # frames are kept apart from the ones timed above.
    stage_sum = {k: 0.0 for k in ivv.STAGES}
    for i in range(args.steps):
        flush.zero_()
        frame(ivv.FLAG_TIMING)
        for k, v in vol.stage_times().items():
            stage_sum[k] += v
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    px_rank = W * H if window is None else FW * FH / world      # rows: the ranks share one frame
    value, ms = aggregate_ranks(ms, px_rank, dist, "cuda")
    if dist:
        dist.barrier()
    k5_ms = stage_sum["integrate"] / args.steps
    k2_ms = stage_sum["intersect"] / args.steps

    # end to end through the C ABI with host buffers (device->host copy inside)
    # (pipelined: ivv_render_to_host_async copies frame i to pinned host
    # memory while frame i + 1 renders; every frame's image reaches the host
    # inside the timed region; the blocking ivv_render_to_host is timed too)
    hosts = [torch.empty((H, W, 4), dtype=torch.float32, pin_memory=True) for _ in range(2)]
    for i in range(2):
        vol.render_to_host(sc.camera, sc.params, W, H, hosts[i], window=window)
        vol.render_to_host_async(sc.camera, sc.params, W, H, hosts[i], window=window)
    vol.wait_host()
    e2e_n = max(3, args.steps)
    t0 = time.perf_counter()
    for i in range(e2e_n):
        vol.render_to_host_async(sc.camera, sc.params, W, H, hosts[i % 2], window=window)
    vol.wait_host()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_n
    e2e_value, e2e_ms = aggregate_ranks(e2e_ms, px_rank, dist, "cuda")
    t0 = time.perf_counter()
    for i in range(e2e_n):
        vol.render_to_host(sc.camera, sc.params, W, H, hosts[i % 2], window=window)
    e2e_sync_ms = (time.perf_counter() - t0) * 1e3 / e2e_n
    e2e_sync_value, e2e_sync_ms = aggregate_ranks(e2e_sync_ms, px_rank, dist, "cuda")

    props = torch.cuda.get_device_properties(local)
    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_fp32 = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    peak_note = ("FP32 lanes: %d SMs x 128 x 2 flop x %.0f MHz (max SM clock)"
                 % (props.multi_processor_count, sm_max))

    sm_load = clocks.get("sm_mhz") if isinstance(clocks, dict) else None
    peak_load = props.multi_processor_count * 128 * 2 * sm_load * 1e6 / 1e12 if sm_load else None

    def roof(kernel, flops, ms, flops_exec=None):
        """flops: the launch's algorithmic work; flops_exec: the work the
        kernels execute where it is larger (the split integration's shading
        pass evaluates J afresh at every sample)."""
        achieved = flops / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
        r = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s",
             "frac": achieved / peak_fp32 if peak_fp32 else None,
             "frac_at_sampled_clock": achieved / peak_load if peak_load else None,
             "traffic": _ncu_traffic(kernel, args.workload),
             "peak_note": peak_note, "flops_per_launch": flops, "ms_per_launch": ms}
        if flops_exec is not None:
            a_x = flops_exec / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
            r["count_rule"] = ("RHS x %d + step attempts x 40 + samples x (100 + the scalar with J at hand)"
                               % F["rhs"])
            r["executed"] = {"flops_per_launch": flops_exec, "achieved": a_x,
                             "frac": a_x / peak_fp32 if peak_fp32 else None,
                             "rule": "as counted, plus the shading pass's fresh J per sample (%d flop), "
                                     "70 per step attempt and 150 per sample" % F["rho_j"]}
        return r

    roofs = sorted([roof("k2_intersect", flops_k2, k2_ms),
                    (roof("stage3_integrate", flops_k5_unit, k5_ms, flops_k5) if flops_k5_unit is not None
                     else roof("stage3_integrate", flops_k5, k5_ms))],
                   key=lambda r: -r["ms_per_launch"])

    cpu_base, rows = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_base, rows = cpu_oracle_sample(sc, label="%dx%d frame" % (W, H))

    # parity of this frame against the oracle (untimed): every pixel of the
    # rows the CPU baseline rendered (the whole frame where it reached stride
    # 1), and the entry/exit points of the same pixels
    parity = pair_err = None
    if rank == 0 and not args.no_parity:
        if rows is None:
            _, rows = cpu_oracle_sample(sc, target_s=6.0, max_stride=32, label="%dx%d frame" % (W, H))
        vol.render(sc.camera, sc.params, W, H, out=out)
        torch.cuda.synchronize()
        parity = image_parity(out.cpu().numpy(), rows)
        # the pair export serves the FP32 / MIXED stages 1-2 only
        pair_err = pair_parity(vol, sc, rows) if prec != 2 else None

    if rank == 0:
        import ctypes
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if window is not None else "weak",
            "vs_baseline": None, "dtype": {0: "f32", 1: "f32+f64", 2: "f64"}[prec], "data": "synthetic",
            "config": {"workload": workload, "width": FW, "height": FH, "rk_tol": sc.params.rk_tol,
                       "ds": sc.params.ds, "supersample_k": sc.params.supersample_k,
                       "l2": "flushed between steps (512 MiB write outside the timed events)",
                       "parallelism": ("row bands of one frame" if window is not None else "replicas")
                       if world > 1 else "single"},
            "stages_ms": {k: v / args.steps for k, v in stage_sum.items()},
            "wall_s_timed_loop": t_wall,
            "gpu_launches": kernels_per_frame(prec, args.rk_method, sc.params.method, sc.params.use_mlp_guess,
                                              len(sc.blocks))
                            * args.steps,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "ms_per_frame": e2e_ms,
                    "api": "ivv_render_to_host_async + ivv_render_to_host_wait (copies overlap the next render)",
                    "blocking": {"value": e2e_sync_value, "ms_per_frame": e2e_sync_ms,
                                 "api": "ivv_render_to_host"},
                    "h2d_bytes_per_step": ctypes.sizeof(ivv.Camera) + ctypes.sizeof(ivv.RenderParams),
                    "d2h_bytes_per_step": W * H * 16},
            "roofline": roofs[0],
            "roofline_kernels": roofs,
            "work": {k: st[k] for k in ("rays", "pairs", "samples", "rk_steps", "rk_rejects", "rhs_evals",
                                        "rho_evals", "fragments", "isect_items", "isect_split", "isect_tests",
                                        "isect_newton")},
            "max_delta_p": st["max_delta_p"],
            "guess_training_s": train_s,
            "parity": parity,
            "entry_exit_parity": pair_err,
            "clocks": clocks,
        }
        if cpu_base:
            line["cpu_baseline"] = cpu_base
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_batch(args):
    """The 64-request batch: one CUDA graph per step (K0, K2, K4, K5 launches
    over all requests), launch shapes from the autotuner's cache."""
    import numpy as np
    import torch

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1404_3363_gb300 import autotune, build as libbuild
    libbuild.build()
    from paper_1404_3363_gb300 import ivv, scenes

    vols, reqs = scenes.batch_requests()
    if args.only_volume is not None:
        reqs = [q for q in reqs if q.volume == args.only_volume]
    if args.requests:
        reqs = reqs[:args.requests]
    gpu = [ivv.volume_for(v) for v in vols]
    items = [(gpu[q.volume], q.camera, q.width, q.height, q.tf) for q in reqs]
    bparams = scenes.RenderParams(rk_tol=args.rk_tol) if args.rk_tol is not None else None
    b = ivv.Batch(items, bparams)
    npix = b.info()["n_pixels"]
    if args.no_autotune:
        tuning, tune_ms, tune_src = b.tuning, None, "default"
    else:
        tuning, tune_ms, tune_src = autotune.tuned(b, items)
    stream = torch.cuda.current_stream()

    b.reset_stats()
    b.render(flags=ivv.FLAG_STATS)
    st = b.stats()
    # the batch pool's volumes share one degree; its shading pass evaluates
    # control-point scalars (cube, beam) and Eq. 23 (bar): counted at the
    # control-point cost, a lower bound on the work
    F = flop_model(scene_degree(vols[0].blocks))
    flops_k5 = k5_flops(st, F, 0)
    b.render(flags=ivv.FLAG_TIMING)
    stages = b.stage_times()

    parity = None
    if rank == 0 and not args.no_parity:
        import oracle
        b.render()
        torch.cuda.synchronize()
        orc = [oracle.OracleVolume(v.blocks, v.scalar_mode) for v in vols]
        max_err, px, nrows = 0.0, 0, 0
        for q, out in zip(reqs, b.outputs):
            img = out.cpu().numpy()
            sc = vols[q.volume]
            sc = type(sc)(sc.name, sc.blocks, sc.scalar_mode, q.tf, q.camera, q.width, q.height,
                          scenes.RenderParams())
            for y in range(5, q.height, 16):            # every 16th row, every pixel of it
                ref = oracle.render(sc, orc[q.volume], window=(0, q.width, y, y + 1))[0]
                max_err = max(max_err, float(np.abs(img[y].astype(np.float64) - ref).max()))
                px += q.width
                nrows += 1
        parity = {"max_rgba_err": max_err, "pixels": px, "rows": nrows,
                  "sample": "every 16th row of every request", "tolerance": 1e-3, "ok": max_err <= 1e-3}

    for _ in range(args.warmup):
        b.render()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(_gpu_id_for_smi(local))
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        ev[i][0].record(stream)
        b.render()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = sum(x.elapsed_time(y) for x, y in ev) / args.steps
    value, ms = aggregate_ranks(ms, npix, dist, "cuda")

    # end to end: graph replay plus every request's image copied to pinned host memory
    hosts = [torch.empty(o.shape, dtype=torch.float32, pin_memory=True) for o in b.outputs]
    e2e_n = max(3, args.steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_n):
        b.render()
        for h_, o in zip(hosts, b.outputs):
            h_.copy_(o, non_blocking=True)
        torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_n
    e2e_value, e2e_ms = aggregate_ranks(e2e_ms, npix, dist, "cuda")

    props = torch.cuda.get_device_properties(local)
    sm_max = float(_peaks().get("sm_max_mhz", 2070.0))
    peak_fp32 = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    k5_ms = stages["integrate"]
    achieved = flops_k5 / (k5_ms * 1e-3) / 1e12
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS["batch64"][2] + (
                           "" if len(reqs) == 64 else " (subset: %d requests)" % len(reqs)) + (
                           ", rk_tol %g" % args.rk_tol if args.rk_tol is not None else ""),
                       "requests": len(reqs), "pixels": npix,
                       "tuning": tuning, "tuning_source": tune_src, "autotune_ms": tune_ms,
                       "l2": "inputs larger than L2 (%.1f GB workspace)" % (b.info()["workspace_bytes"] / 1e9),
                       "parallelism": "replicas" if world > 1 else "single"},
            "stages_ms_timed_render": stages,
            "gpu_launches": BATCH_KERNELS * args.steps,
            "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_batch": e2e_ms, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": npix * 16},
            "roofline": {"bound": "alu", "kernel": "stage3_integrate (batched)", "achieved": achieved,
                         "peak": peak_fp32, "unit": "TFLOP/s", "frac": achieved / peak_fp32, "traffic": None,
                         "flops_per_launch": flops_k5, "ms_per_launch": k5_ms},
            "work": {k: st[k] for k in ("rays", "pairs", "samples", "rk_steps", "rk_rejects", "rhs_evals",
                                        "rho_evals", "fragments", "isect_items", "isect_split", "isect_tests",
                                        "isect_newton")},
            "parity": parity,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--ref-stride", type=int, default=96)
    ap.add_argument("--workload", default="bar1080", choices=sorted(WORKLOADS) + sorted(LEARNED_WORKLOADS))
    ap.add_argument("--requests", type=int, default=0, help="batch64: keep the first N requests (0: all)")
    ap.add_argument("--only-volume", type=int, default=None, help="batch64: keep the requests of one volume")
    ap.add_argument("--no-autotune", action="store_true", help="batch64: default launch shapes")
    ap.add_argument("--split", default="replicas", choices=["replicas", "rows"],
                    help="N > 1: every rank renders its own frame (replicas, weak scaling) or a band of rows of "
                         "one frame (strong scaling)")
    ap.add_argument("--rk-method", type=int, default=0, choices=range(8),
                    help="single-frame workloads: 0 BS3(2) with error control, 1-6 the explicit fixed-step "
                         "family, 7 implicit Euler")
    ap.add_argument("--c", type=float, default=None, help="single-frame workloads: the pull-back constant c "
                                                           "of the ray field (Eq. 10; default 1)")
    ap.add_argument("--rk-tol", type=float, default=None,
                    help="single-frame workloads: the embedded pair's local error bound (default: the workload's)")
    ap.add_argument("--guess-samples", type=int, default=1 << 20,
                    help="learned workloads: forward-map samples per block the guess network trains on")
    ap.add_argument("--guess-epochs", type=int, default=8, help="learned workloads: training epochs")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
