"""Benchmark: direct volume rendering, forward + backward, on synthetic HI-like
cubes through the C ABI (libvr.so).

Default workload (one "step"): a 1024^3 float32 HI-like cube (noise + 2000
Gaussian blobs + 200 rotating-disk sources) resident in HBM as bricks; eight
1920x1080 perspective orbit views rendered by ONE batched persistent launch
(CUDA graph), step 1 voxel, early termination at opacity 0.99; then the
adjoint of each view (table + voxel gradients, accumulated over the views)
against a fixed seeded dL/dI.

value = forward-composited samples of the 8 views / step time (Gsamples/s).
Also reported: 1080p frames/s for fwd+bwd, forward-only rates (batched and
the plain FP32 single-view vr_render form), pixel error against the FP64
oracle on sampled rows, the roofline object of the dominant kernel, the
oracle timed on the host cores, and the end-to-end rate with host buffers.

--impl reference times the FP64 oracle (the only reference this method has)
on a bounded sample of the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "DVR Gsamples/s and 1080p fps fwd+bwd on 1 GB300 vs plain FP32 at stated px error"
UNIT = "Gsamples/s"
GATHER_BYTES_F32 = 8 * 4          # algorithmic bytes of one sample: 8 trilinear corners x 4 B


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def gather_rate_frac(gsamples_per_s: float, bytes_per_voxel: int) -> float:
    """Fraction of the HBM gather rate R = BW / (8 s): samples per second
    times the trilinear footprint's 8 s bytes, over the measured copy
    bandwidth."""
    return gsamples_per_s * 8 * bytes_per_voxel / measured_peaks()[0]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def kernel_sources_sha256() -> str:
    """Digest of the CUDA sources, to tell whether recorded counters still
    describe the kernels being run."""
    import hashlib
    d = os.path.join(ROOT, "paper_1211_4896_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h", ".cpp")):
            with open(os.path.join(d, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def recorded_traffic(kernel: str):
    """DRAM bytes (read + write) of one call of `kernel` on this workload (the
    multi-view backward: its eight launches), from the ncu capture summarised
    in profiles/traffic_scale_1024.json; None when the CUDA sources have
    changed since that capture."""
    p = os.path.join(ROOT, "profiles", "traffic_scale_1024.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    if rec.get("sources_sha256") != kernel_sources_sha256():
        return None
    v = rec.get("dram_bytes_per_call", {}).get(kernel)
    return None if v is None else float(v)


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        """Ends the sampling; returns the summary of this region (None
        without samples).  The raw samples stay in self.raw."""
        self.raw = []
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm, mx = float(parts[1]), float(parts[2])
                except ValueError:
                    continue
                self.raw.append((sm, mx, {n for n, v in zip(names, parts[5:9]) if v.lower() == "active"}))
        os.unlink(self.path)
        return self.summarize(self.raw)

    @staticmethod
    def summarize(raw):
        if not raw:
            return None
        return {"sm_mhz": statistics.median(r[0] for r in raw), "sm_max_mhz": max(r[1] for r in raw),
                "reasons": sorted(set().union(*(r[2] for r in raw))), "samples": len(raw)}


class ClockLog:
    """Clock samples of every timed region of one workload line (the
    secondary workloads time several regions; each is sampled while it runs)."""

    def __init__(self):
        self.raw = []

    def sampler(self):
        return ClockSampler(_env_int("LOCAL_RANK", 0))

    def add(self, sampler):
        sampler.stop()
        self.raw += sampler.raw

    def take(self):
        out, self.raw = ClockSampler.summarize(self.raw), []
        return out


CLOCKS = ClockLog()


# ---------------------------------------------------------------------------
# Ceilings of a workload (measurement only; none of this is on the render path)
# ---------------------------------------------------------------------------

def footprint_voxels(torch, dims, cam, step, nsamples, max_bitmap_bytes=2 << 30):
    """Distinct voxels touched by the trilinear footprints of one view's
    composited samples (the view's compulsory voxel set).  Each pixel's ray
    is re-derived in float64 with the renderer's camera conventions (basis
    f, r = f x up, u = r x f; pixel centres; slab clip to the closed box
    [0, n-1]; perspective rays from the eye), its first nsamples[j, i]
    samples are placed at t_in + (k + 1/2) step, their cells (clamped corner
    floor(p)) are marked in a bitmap and the bitmap is dilated by one voxel
    towards +x, +y and +z (a cell's eight corners).  Unit spacing, origin 0.
    Large grids are counted in slabs of cells along z."""
    dev = nsamples.device
    f64 = torch.float64
    nx, ny, nz = (int(d) for d in dims)
    H, W = int(cam["height"]), int(cam["width"])
    f = torch.tensor(cam["forward"], dtype=f64, device=dev)
    f = f / f.norm()
    up = torch.tensor(cam["up"], dtype=f64, device=dev)
    r = torch.linalg.cross(f, up)
    r = r / r.norm()
    u = torch.linalg.cross(r, f)
    jj, ii = torch.meshgrid(torch.arange(H, device=dev, dtype=f64), torch.arange(W, device=dev, dtype=f64),
                            indexing="ij")
    sx = ((ii + 0.5) / W) * 2.0 - 1.0
    sy = 1.0 - ((jj + 0.5) / H) * 2.0
    aspect = W / H
    eye = torch.tensor(cam["eye"], dtype=f64, device=dev)
    if cam["kind"] == 0:
        hh = 0.5 * cam["ortho_height"]
        o = eye + (sx * hh * aspect)[..., None] * r + (sy * hh)[..., None] * u
        d = f.expand(H, W, 3)
        t0 = torch.full((H, W), -math.inf, dtype=f64, device=dev)
    else:
        th = math.tan(math.radians(cam["fov_y_deg"]) / 2.0)
        d = f + (sx * th * aspect)[..., None] * r + (sy * th)[..., None] * u
        d = d / d.norm(dim=-1, keepdim=True)
        o = eye.expand(H, W, 3)
        t0 = torch.zeros((H, W), dtype=f64, device=dev)
    t1 = torch.full((H, W), math.inf, dtype=f64, device=dev)
    hi = torch.tensor([nx - 1, ny - 1, nz - 1], dtype=f64, device=dev)
    with torch.no_grad():
        for a in range(3):
            da = d[..., a]
            inv = 1.0 / da
            ta, tb = (0.0 - o[..., a]) * inv, (hi[a] - o[..., a]) * inv
            t0 = torch.where(da != 0, torch.maximum(t0, torch.minimum(ta, tb)), t0)
            t1 = torch.where(da != 0, torch.minimum(t1, torch.maximum(ta, tb)), t1)
        n = nsamples.to(torch.int64).reshape(-1)
        order = torch.argsort(n, descending=True)
        n = n[order]
        o = o.reshape(-1, 3)[order]
        d = d.reshape(-1, 3)[order]
        t0 = t0.reshape(-1)[order]
        ncx, ncy, ncz = nx - 1, ny - 1, nz - 1
        slab = max(1, min(ncz, max_bitmap_bytes // max(1, ncx * ncy)))
        total = 0
        carry = None
        for z_lo in range(0, ncz, slab):
            z_hi = min(ncz, z_lo + slab)
            cells = torch.zeros((z_hi - z_lo) * ncy * ncx, dtype=torch.bool, device=dev)
            live = int((n > 0).sum())
            k = 0
            while live > 0:
                t = t0[:live] + (k + 0.5) * step
                p = o[:live] + t[:, None] * d[:live]
                c = torch.floor(p).to(torch.int64)
                cx = c[:, 0].clamp(0, ncx - 1)
                cy = c[:, 1].clamp(0, ncy - 1)
                cz = c[:, 2].clamp(0, ncz - 1)
                m = (cz >= z_lo) & (cz < z_hi)
                cells[((cz[m] - z_lo) * ncy + cy[m]) * ncx + cx[m]] = True
                k += 1
                while live > 0 and int(n[live - 1]) <= k:
                    live -= 1
            cells = cells.view(z_hi - z_lo, ncy, ncx)
            # voxel layers [z_lo, z_hi] touched by this slab's cells; layer z_lo
            # also takes the previous slab's top layer, layer z_hi is carried
            # to the next slab (the last slab counts it)
            vox = torch.zeros((z_hi - z_lo + 1, ny, nx), dtype=torch.bool, device=dev)
            for dz in (0, 1):
                for dy in (0, 1):
                    for dx in (0, 1):
                        vox[dz:dz + z_hi - z_lo, dy:dy + ncy, dx:dx + ncx] |= cells
            if carry is not None:
                vox[0] |= carry
            if z_hi < ncz:
                total += int(vox[:-1].sum())
                carry = vox[-1].clone()
            else:
                total += int(vox.sum())
            del cells, vox
        return total


def issue_per_sample(kernel: str):
    """Warp instructions issued per composited sample for `kernel`, measured
    with ncu on the small profile cases (profiles/issue_per_sample.json; the
    case of each figure is recorded there), or None."""
    p = os.path.join(ROOT, "profiles", "issue_per_sample.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    if rec.get("sources_sha256") != kernel_sources_sha256():
        return None
    v = rec.get("warp_inst_per_sample", {}).get(kernel)
    return None if v is None else float(v)


def ceilings(samples, seconds, bytes_per_voxel, b_alg, kernel, sm_mhz):
    """The three rates that bound a pass of the march (samples per second),
    the one that binds, and where the achieved rate stands:
      gather      BW / (8 s): every sample's eight corners from HBM, no reuse;
      compulsory  samples BW / B_alg: each voxel any footprint touches read
                  from HBM once (B_alg = s x touched voxels);
      issue       SMs x 4 warp instructions per clock / instructions per
                  sample (measured on the profile case of this kernel)."""
    bw = measured_peaks()[0] * 1e9
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = {"gather_gs": bw / (8 * bytes_per_voxel) / 1e9}
    if b_alg:
        out["compulsory_gs"] = samples * bw / b_alg / 1e9
        out["b_alg_bytes"] = b_alg
        out["b_alg_per_sample"] = b_alg / samples
    ips = issue_per_sample(kernel)
    if ips and sm_mhz:
        out["issue_gs"] = sms * 4 * sm_mhz * 1e6 / ips / 1e9
        out["warp_inst_per_sample"] = ips
    rates = {k[:-3]: v for k, v in out.items() if k.endswith("_gs")}
    out["binding"] = min(rates, key=rates.get)
    out["achieved_gs"] = samples / seconds / 1e9
    out["achieved_frac_of_binding"] = out["achieved_gs"] / rates[out["binding"]]
    return out


# ---------------------------------------------------------------------------
# Reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_step(host_cube, cams, tf_np, pre, rows_per_view, grad_rows):
    """One bounded oracle step: forward + backward (table gradient) of
    ``rows_per_view`` rows of every view.  Returns (samples, seconds)."""
    import oracle
    t0 = time.perf_counter()
    samples = 0
    for vi, cam in enumerate(cams):
        H = cam["height"]
        for q in range(rows_per_view):
            r = (H // 2 - rows_per_view // 2 + q + 37 * vi) % H
            o = oracle.render(host_cube, cam, tf_np, synth.TF_VMIN, synth.TF_VMAX, pre["step"], pre["ert"],
                              rows=(r, r + 1))
            samples += int(o["n_used"][r].sum())
            g = np.zeros((H, cam["width"], 4))
            g[r] = grad_rows[q % len(grad_rows)]
            oracle.render_backward(host_cube, cam, tf_np, synth.TF_VMIN, synth.TF_VMAX, pre["step"], g,
                                   ert=pre["ert"], want_vox=False, rows=(r, r + 1))
    return samples, time.perf_counter() - t0


def adaptive_rows(host_cube, cams, tf_np, pre, grad_rows, target_s):
    """Rows per view so that one oracle step takes about target_s seconds."""
    _, t1 = oracle_step(host_cube, cams, tf_np, pre, 1, grad_rows)
    return int(min(64, max(1, round(target_s / max(t1, 1e-3)))))


def make_cube(pre, device):
    return synth.hi_cube(pre["dims"], pre["n_blobs"], pre["n_disks"], pre["seed"], device=device)


def run_reference(args, rank):
    if rank != 0:
        return 0
    import oracle
    import torch
    oracle.build()
    pre = synth.preset_scale_1024()
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    host = make_cube(pre, dev).cpu().numpy()
    tf_np = synth.tf_ramp(256)
    cams = pre["cameras"]
    rng = np.random.default_rng(0)
    grad_rows = [rng.normal(size=(cams[0]["width"], 4)) for _ in range(4)]
    rows = adaptive_rows(host, cams, tf_np, pre, grad_rows, target_s=4.0)
    for _ in range(args.warmup):
        oracle_step(host, cams, tf_np, pre, rows, grad_rows)
    tot_s, tot_t = 0, 0.0
    for _ in range(args.steps):
        s, t = oracle_step(host, cams, tf_np, pre, rows, grad_rows)
        tot_s += s
        tot_t += t
    value = tot_s / tot_t / 1e9
    cores = os.cpu_count()
    sample = ("per step: %d row(s) of each of the 8 views (1920 rays/row), FP64 forward + backward "
              "(table gradient; the voxel gradient is not computed)" % rows)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "scale_1024 (sampled rows)", "views": 8, "image": [1920, 1080]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------

def reduce_over_ranks(ms: float, samples: int, device) -> tuple:
    """Whole-job figures across ranks: the slowest rank's time and the sum of
    every rank's composited samples (each rank renders its own views)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, samples
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    n = torch.tensor([samples], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1211_4896_gb300 as P
    from paper_1211_4896_gb300 import _lib as L

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    pre = synth.preset_scale_1024()
    cube = make_cube(pre, dev)
    vol = P.Volume(cube, "f32")
    host_cube = cube.cpu().numpy() if rank == 0 else None
    del cube
    torch.cuda.empty_cache()
    cams = pre["cameras"]
    nv = len(cams)
    H, W = cams[0]["height"], cams[0]["width"]
    tf_np = synth.tf_ramp(256)
    tf = torch.from_numpy(tf_np).to(dev)
    vmin, vmax, step, ert = synth.TF_VMIN, synth.TF_VMAX, pre["step"], pre["ert"]
    outs = [torch.empty((H, W, 4), device=dev) for _ in range(nv)]
    nss = [torch.empty((H, W), device=dev, dtype=torch.int32) for _ in range(nv)]
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234)
    grads = [torch.randn((H, W, 4), device=dev, generator=gen) for _ in range(nv)]
    grad_tf = torch.empty((256, 4), device=dev, dtype=torch.float64)
    nz, ny, nx = vol.shape
    grad_vox = torch.empty((nz, ny, nx), device=dev, dtype=torch.float32)
    stream = torch.cuda.current_stream()
    s_ptr = int(stream.cuda_stream)

    jobs = [dict(vol=vol, cam=c, tf=tf, vmin=vmin, vmax=vmax, step=step, ert=ert, out=o, nsamples=n)
            for c, o, n in zip(cams, outs, nss)]
    cjobs = P.render_batched(jobs, use_graph=True)          # builds the plan + graph
    opts = L.vr_batch_opts(1, 8, 4, 0)
    ccams = [L.make_camera(c) for c in cams]
    # the batched call launches one kernel per brick layout its views read; the
    # multi-view backward one kernel per view and one FP64 row sum
    groups = len({L.vr_view_layout(vol.handle, cc) for cc in ccams})
    gviews = [L.vr_grad_view(cc, o.data_ptr(), n.data_ptr(), g.data_ptr())
              for cc, o, n, g in zip(ccams, outs, nss, grads)]
    cpar = L.make_params(tf.data_ptr(), 256, vmin, vmax, step, ert)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def fwd():
        L.vr_render_batched(cjobs, opts, s_ptr)

    def bwd():              # the loss summed over the 8 views: one multi-view call
        L.vr_render_backward_views(vol.handle, gviews, cpar, grad_tf.data_ptr(), grad_vox.data_ptr(), 0, s_ptr)

    fwd_ev, bwd_ev = [], []

    def step_fn(record):
        if record:
            e0, e1 = ev(), ev()
            e0.record(stream)
        fwd()
        if record:
            e1.record(stream)
            fwd_ev.append((e0, e1))
        if record:
            b0, b1 = ev(), ev()
            b0.record(stream)
        bwd()
        if record:
            b1.record(stream)
            bwd_ev.append((b0, b1))

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step_fn(False)
    torch.cuda.synchronize()
    samples_per_step = int(sum(int(n.sum().item()) for n in nss))

    clocks = ClockSampler(local_rank)
    barrier()
    clocks.start()
    t_start, t_end = ev(), ev()
    t_start.record(stream)
    for _ in range(args.steps):
        step_fn(True)
    t_end.record(stream)
    barrier()
    clk = clocks.stop()
    ms = t_start.elapsed_time(t_end) / args.steps
    fwd_ms = statistics.mean(a.elapsed_time(b) for a, b in fwd_ev)
    bwd_ms = statistics.mean(a.elapsed_time(b) for a, b in bwd_ev)           # the 8 views
    ms_max, samples_all = reduce_over_ranks(ms, samples_per_step, dev)
    value = samples_all / (ms_max * 1e-3) / 1e9

    # ---- forward-only rates (batched graph and plain single-view form) -------------
    e0, e1 = ev(), ev()
    torch.cuda.synchronize()
    e0.record(stream)
    reps = max(3, args.steps)
    for _ in range(reps):
        fwd()
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_only_ms = e0.elapsed_time(e1) / reps
    view_ms = []
    for v in range(nv):
        a, b = ev(), ev()
        L.vr_render(vol.handle, ccams[v], cpar, outs[v].data_ptr(), nss[v].data_ptr(), s_ptr)   # warm
        a.record(stream)
        for _ in range(3):
            L.vr_render(vol.handle, ccams[v], cpar, outs[v].data_ptr(), nss[v].data_ptr(), s_ptr)
        b.record(stream)
        torch.cuda.synchronize()
        view_ms.append(a.elapsed_time(b) / 3)
    plain_ms = sum(view_ms)
    p75 = float(np.percentile(view_ms, 75))

    # ---- end to end through the C ABI with host buffers ------------------------------
    pin_tf = torch.from_numpy(tf_np).pin_memory()
    pin_g = [g.cpu().pin_memory() for g in grads]
    pin_out = [torch.empty((H, W, 4), pin_memory=True) for _ in range(nv)]
    pin_gtf = torch.empty((256, 4), dtype=torch.float64, pin_memory=True)
    h2d = pin_tf.numel() * 4 + sum(g.numel() * 4 for g in pin_g)
    d2h = sum(o.numel() * 4 for o in pin_out) + pin_gtf.numel() * 8

    # The step's host copies run on a copy stream beside the kernels: the
    # gradient images go up while the forward runs (the backward waits for
    # them), the rendered images come down while the backward runs (the next
    # forward waits for them), the table gradient after the backward.
    copy_stream = torch.cuda.Stream(device=dev)
    ev_bwd, ev_d2h = torch.cuda.Event(), torch.cuda.Event()
    ev_bwd.record(stream)
    ev_d2h.record(stream)

    def e2e_step():
        ev_h2d, ev_fwd = torch.cuda.Event(), torch.cuda.Event()
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(ev_bwd)             # the last backward has read the gradients
            for g, pg in zip(grads, pin_g):
                g.copy_(pg, non_blocking=True)
            ev_h2d.record(copy_stream)
        stream.wait_event(ev_d2h)                      # the last images have been read out
        tf.copy_(pin_tf, non_blocking=True)
        fwd()
        ev_fwd.record(stream)
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(ev_fwd)
            for o, po in zip(outs, pin_out):
                po.copy_(o, non_blocking=True)
            ev_d2h.record(copy_stream)
        stream.wait_event(ev_h2d)
        bwd()
        ev_bwd.record(stream)
        pin_gtf.copy_(grad_tf, non_blocking=True)

    e2e_step()
    barrier()
    a, b = ev(), ev()
    a.record(stream)
    for _ in range(args.steps):
        e2e_step()
    stream.wait_event(ev_d2h)                          # the last step's images are on the host
    b.record(stream)
    barrier()
    e2e_ms, _ = reduce_over_ranks(a.elapsed_time(b) / args.steps, samples_per_step, dev)
    e2e_value = samples_all / (e2e_ms * 1e-3) / 1e9

    # ---- pixel error against the FP64 oracle: three rows of every view ----------------
    px = None
    cpu = None
    if rank == 0:
        import oracle
        from oracle.parity import compare_pixels
        oracle.build()
        fwd()
        torch.cuda.synchronize()
        res = []
        for v, cam in enumerate(cams):
            img, ns = outs[v].cpu().numpy(), nss[v].cpu().numpy()
            rows = [H // 2 - 100 + 7 * v, H // 2 + 7 * v, H // 2 + 100 + 7 * v]
            ref = _oracle_rows(oracle, host_cube, cam, tf_np, vmin, vmax, step, ert, rows)
            res.append(compare_pixels(img, ns, ref, PX_TOL_F32, rows=rows, raise_on_fail=False))
        px = _merge_px(res, "FP64 oracle, rows H/2-100+7v, H/2+7v, H/2+100+7v of each view v = 0..7 (batched "
                            "forward); count differences allowed only on an oracle-reported tie")
        # ---- CPU baseline: the oracle on a bounded sample -------------------------------
        rng = np.random.default_rng(0)
        grad_rows = [rng.normal(size=(W, 4)) for _ in range(4)]
        nrows = adaptive_rows(host_cube, cams, tf_np, pre, grad_rows, target_s=12.0)
        s, t = oracle_step(host_cube, cams, tf_np, pre, nrows, grad_rows)
        cpu = {"value": s / t / 1e9, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": "%d row(s) of each of the 8 views (1920 rays per row), FP64 forward + backward "
                         "(table gradient only), %d composited samples in %.1f s" % (nrows, s, t)}

    # ---- roofline of the dominant kernel ---------------------------------------------
    peak, peak_kind = measured_peaks()
    if bwd_ms >= fwd_ms:
        dom, dom_key, dom_ms, per = ("bwd_kernel (one multi-view call: 8 launches over two streams; timed with "
                                     "its scratch clear and FP64 row sum)", "bwd_kernel", bwd_ms, samples_per_step)
    else:
        dom, dom_key, dom_ms, per = "batched_kernel (8 views, one launch)", "batched_kernel", fwd_ms, samples_per_step
    achieved = per * GATHER_BYTES_F32 / (dom_ms * 1e-3) / 1e9
    traffic = recorded_traffic(dom_key)
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
            "per_unit": "8 x 4 B trilinear gathers per composited sample"}
    # the compulsory voxel set of every view (measurement only, after the timed region)
    b_alg = 4 * sum(footprint_voxels(torch, vol.shape[::-1], c, step, n) for c, n in zip(cams, nss)) if rank == 0 \
        else None
    sm_mhz = clk["sm_mhz"] if clk else None
    ceil = {"fwd_batched": ceilings(samples_per_step, fwd_only_ms * 1e-3, 4, b_alg, "batched_kernel<float>", sm_mhz),
            "bwd": ceilings(samples_per_step, bwd_ms * 1e-3, 4, b_alg, "bwd_kernel<float>", sm_mhz)}
    if traffic and b_alg:
        roof["waste_ratio"] = traffic / b_alg      # DRAM bytes of the kernel's launches / compulsory bytes

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "scale_1024: 1024^3 f32 HI-like cube (noise + 2000 blobs + 200 disks), "
                                   "8 perspective orbit views at 1920x1080, step 1 voxel, ERT 0.99; "
                                   "fwd = one batched graph launch of the 8 views, bwd = table + voxel "
                                   "gradients of the loss summed over the 8 views (one multi-view call)",
                       "views": nv, "image": [W, H], "samples_per_step": samples_per_step,
                       "l2": "inputs larger than L2 (bricked cube %.2f GB)" % (vol.info["bytes"] / 1e9),
                       "parallelism": "views replicated per GPU" if world > 1 else "1 GPU"},
            "fps_fwd_bwd": nv * world / (ms_max * 1e-3),
            "fwd": {"batched_gsamples_per_s": samples_per_step / (fwd_only_ms * 1e-3) / 1e9,
                    "batched_ms_8_views": fwd_only_ms,
                    "plain_fp32_single_view_gsamples_per_s": samples_per_step / (plain_ms * 1e-3) / 1e9,
                    "plain_fp32_view_ms_p75": p75, "fps_p75": 1e3 / p75},
            "bwd": {"ms_8_views": bwd_ms, "bwd_over_fwd": bwd_ms / fwd_ms},
            "px_err": px, "roofline": roof, "ceilings": ceil, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "copies": "pinned host buffers through a copy stream: each step's gradient images go up "
                              "during its forward, its images come down during its backward, its table "
                              "gradient after it; all inside the timed region"},
            "gpu_launches": args.steps * (groups + nv + 1), "clocks": clk}
    if rank == 0:
        print(json.dumps(line))
    vol.close()
    if dist is not None:
        dist.destroy_process_group()
    if px is not None and not px["passed"]:
        print("bench: the pixel-error check against the oracle failed: %s" % px.get("problems"), file=sys.stderr)
        return 1
    return 0


# ---------------------------------------------------------------------------
# Other workloads (reported lines; the default workload above is the
# benchmark's contract line)
# ---------------------------------------------------------------------------

def _time_ms(torch, fn, reps, min_s=0.6):
    """Mean CUDA-event time of fn over at least `reps` calls and at least
    min_s seconds (so that the clock sampler sees the region), after one
    untimed call; SM clocks are sampled during the timed calls (CLOCKS)."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    e0.record()
    fn()
    e1.record()
    torch.cuda.synchronize()
    once = max(e0.elapsed_time(e1), 1e-3)
    reps = max(reps, int(math.ceil(min_s * 1e3 / once)))
    clk = CLOCKS.sampler()
    clk.start()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    CLOCKS.add(clk)
    return e0.elapsed_time(e1) / reps


def _emit(line):
    """Prints one workload line with the clock record of its timed regions."""
    line["clocks"] = CLOCKS.take()
    print(json.dumps(line))


PX_TOL_F32 = 1e-4        # max abs pixel error, float32 storage
PX_TOL_HALF = 2e-3       # 16-bit storage, against the oracle on the float32 cube


def _oracle_rows(oracle, host, cam, tf_np, vmin, vmax, step, ert, rows):
    """The oracle's render of the given rows (other rows stay zero)."""
    ref = {}
    for r in rows:
        o = oracle.render(host, cam, tf_np, vmin, vmax, step, ert, rows=(r, r + 1))
        for k, v in o.items():
            ref.setdefault(k, np.zeros_like(v))[r] = v[r]
    return ref


def _merge_px(results, against):
    """One pixel-error record from several compare_pixels results."""
    n = sum(r["pixels"] for r in results)
    out = {"max_abs": max(r["max_abs"] for r in results),
           "mean_abs": sum(r["mean_abs"] * r["pixels"] for r in results) / max(n, 1),
           "pixels": n, "excluded_ties": sum(r["excluded_ties"] for r in results),
           "off_tie": sum(r["off_tie"] for r in results), "passed": all(r["passed"] for r in results),
           "against": against}
    probs = [p for r in results for p in r.get("problems", [])]
    if probs:
        out["problems"] = probs[:4]
    return out


def _px_err(img, ns, ref, rows, tol=PX_TOL_F32):
    from oracle.parity import compare_pixels
    return compare_pixels(img, ns, ref, tol, rows=rows, raise_on_fail=False)


def run_plain_128(args):
    """128^3 f32, orthographic along +z, 256^2, step 0.5, no early termination."""
    import torch
    import oracle
    import paper_1211_4896_gb300 as P
    pre = synth.preset_plain_128()
    dev = torch.device("cuda")
    cube = synth.hi_cube(pre["dims"], pre["n_blobs"], pre["n_disks"], pre["seed"])
    vol = P.Volume(cube.to(dev), "f32")
    tf_np = synth.tf_ramp(256)
    tf = torch.from_numpy(tf_np).to(dev)
    cam = pre["cameras"][0]
    out = torch.empty((256, 256, 4), device=dev)
    ns = torch.empty((256, 256), device=dev, dtype=torch.int32)
    f = lambda: P.render(vol, cam, tf, synth.TF_VMIN, synth.TF_VMAX, pre["step"], pre["ert"], out=out, nsamples=ns)  # noqa
    ms = _time_ms(torch, f, max(20, args.steps))
    samples = int(ns.sum())
    t0 = time.perf_counter()
    ref = oracle.render(cube.numpy(), cam, tf_np, synth.TF_VMIN, synth.TF_VMAX, pre["step"], pre["ert"])
    t_cpu = time.perf_counter() - t0
    err = _px_err(out.cpu().numpy(), ns.cpu().numpy(), ref, range(256))
    line = {"workload": "plain_128", "gsamples_per_s": samples / ms / 1e6, "ms": ms, "samples": samples,
            "roofline_frac": gather_rate_frac(samples / ms / 1e6, 4),
            "px_err": err, "oracle_gsamples_per_s": samples / t_cpu / 1e9, "oracle_cores": os.cpu_count()}
    b_alg = 4 * footprint_voxels(torch, pre["dims"], cam, pre["step"], ns)
    clk = dict(CLOCKS.raw and ClockSampler.summarize(CLOCKS.raw) or {})
    line["ceilings"] = ceilings(samples, ms * 1e-3, 4, b_alg, "fwd_kernel<float>@plain_128", clk.get("sm_mhz"))
    _emit(line)


def run_precision_4096(args):
    """4096x4096x1024 HI-like cube (blob and disk densities of the smaller
    workloads), stored f32 / f16 / bf16; four 1080p perspective views, step 1,
    ERT 0.99; pixel error against the FP64 oracle on a 256^3 crop."""
    import torch
    import oracle
    import paper_1211_4896_gb300 as P
    dev = torch.device("cuda")
    dims = (4096, 4096, 1024)
    nb = int(round(20 * (4096 * 4096 * 1024) / 128 ** 3))
    nd = int(round(200 * (4096 * 4096 * 1024) / 1024 ** 3))
    cube = synth.hi_cube(dims, nb, nd, seed=3, device=dev)
    cams = synth.orbit_cameras(dims, 4, 40.0, 1920, 1080)
    tf_np = synth.tf_ramp(256)
    tf = torch.from_numpy(tf_np).to(dev)
    res = {"workload": "precision_4096", "dims": dims, "blobs": nb, "disks": nd}
    crop = cube[384:640, 1920:2176, 1920:2176].contiguous()          # 256^3 crop (z, y, x)
    crop_np = crop.cpu().numpy()
    crop_cams = synth.orbit_cameras((256, 256, 256), 4, 40.0, 1920, 1080, start_deg=30.0)
    rows = [300 + 60 * q for q in range(8)]
    refs = []
    for cam in crop_cams:
        r = {}
        for row in rows:
            o = oracle.render(crop_np, cam, tf_np, synth.TF_VMIN, synth.TF_VMAX, 1.0, 0.99, rows=(row, row + 1))
            for k, v in o.items():
                r.setdefault(k, np.zeros_like(v))[row] = v[row]
        refs.append(r)
    base = None
    b_alg_vox = None
    from paper_1211_4896_gb300 import _lib as L
    for store in ("f32", "f16", "bf16"):
        vol = P.Volume(cube, store)
        outs = [torch.empty((1080, 1920, 4), device=dev) for _ in cams]
        nss = [torch.empty((1080, 1920), device=dev, dtype=torch.int32) for _ in cams]

        def f():
            for c, o, n in zip(cams, outs, nss):
                P.render(vol, c, tf, synth.TF_VMIN, synth.TF_VMAX, 1.0, 0.99, out=o, nsamples=n)
        ms = _time_ms(torch, f, 3)
        samples = sum(int(n.sum()) for n in nss)
        per_view = []
        for c, o, n in zip(cams, outs, nss):
            ms_v = _time_ms(torch, lambda: P.render(vol, c, tf, synth.TF_VMIN, synth.TF_VMAX, 1.0, 0.99, out=o,
                                                    nsamples=n), 3, min_s=0.2)
            per_view.append({"ms": ms_v, "rays_hit": int((n > 0).sum()), "samples": int(n.sum())})
        layouts = [L.vr_view_layout(vol.handle, L.make_camera(c)) for c in cams]
        vol.close()
        torch.cuda.empty_cache()
        if b_alg_vox is None:       # the same samples for every storage type
            b_alg_vox = sum(footprint_voxels(torch, dims, c, 1.0, n, max_bitmap_bytes=24 << 30)
                            for c, n in zip(cams, nss))
            torch.cuda.empty_cache()
        cvol = P.Volume(crop, store)
        errs = []
        for cam, ref in zip(crop_cams, refs):
            img, ns = P.render(cvol, cam, tf, synth.TF_VMIN, synth.TF_VMAX, 1.0, 0.99)
            errs.append(_px_err(img.cpu().numpy(), ns.cpu().numpy(), ref, rows,
                                PX_TOL_F32 if store == "f32" else PX_TOL_HALF))
        cvol.close()
        gs = samples / ms / 1e6
        base = base or gs
        eb = 4 if store == "f32" else 2
        kern = "fwd_kernel<float>@sparse" if store == "f32" else (
            "fwd_kernel<Blocked<16-bit>>@sparse" if min(layouts) >= 6 else "fwd_kernel<16-bit>@sparse")
        clk = ClockSampler.summarize(CLOCKS.raw) or {}
        res[store] = {"gsamples_per_s": gs, "ms_4_views": ms, "fps": 4e3 / ms, "vs_f32": gs / base,
                      "roofline_frac": gather_rate_frac(gs, eb), "layouts": layouts, "per_view": per_view,
                      "ceilings": ceilings(samples, ms * 1e-3, eb, eb * b_alg_vox, kern, clk.get("sm_mhz")),
                      "bricked_gb": vol.info["bytes"] / 1e9,
                      "crop_px_err": _merge_px(errs, "FP64 oracle on the float32 256^3 crop, rows %s of its 4 "
                                                     "views" % rows)}
        torch.cuda.empty_cache()
    _emit(res)


def run_batch_64(args):
    """64 uneven f16 HI-like cubes (64^3 .. 512x512x1024), each with its own
    perspective camera, image (512^2 .. 1024^2) and random piecewise-linear
    table: one persistent CUDA-graph launch against 64 vr_render launches."""
    import torch
    import paper_1211_4896_gb300 as P
    from paper_1211_4896_gb300 import _lib as L
    dev = torch.device("cuda")
    dims_list = synth.batch_dims(seed=4, n=64)
    jobs = []
    for q, dims in enumerate(dims_list):
        vox = dims[0] * dims[1] * dims[2]
        cube = synth.hi_cube(dims, max(1, int(round(20 * vox / 128 ** 3))), max(0, int(round(200 * vox / 1024 ** 3))),
                             seed=4000 + q, device=dev)
        vol = P.Volume(cube, "f16")
        del cube
        W, H = synth.batch_image_size(seed=5000 + q)
        cam = synth.camera_random_persp(dims, seed=6000 + q, width=W, height=H)
        tf = torch.from_numpy(synth.tf_random_pwl(seed=7000 + q)).to(dev)
        jobs.append(dict(vol=vol, cam=cam, tf=tf, vmin=-3.0, vmax=50.0, step=1.0, ert=0.99,
                         out=torch.empty((H, W, 4), device=dev),
                         nsamples=torch.empty((H, W), device=dev, dtype=torch.int32)))
    torch.cuda.empty_cache()
    s = int(torch.cuda.current_stream().cuda_stream)
    # the autotuner: brick size (volumes re-bricked on the device), tile shape,
    # CTAs per SM and warps per tile
    opts, brick, tuned = P.autotune_batched_bricks(jobs, brick_sizes=(16, 32, 64))
    cj = P.render_batched(tuned, opts=opts)
    t_graph = _time_ms(torch, lambda: L.vr_render_batched(cj, opts, s), max(5, args.steps))
    ccams = [(j["vol"].handle, L.make_camera(j["cam"]),
              L.make_params(j["tf"].data_ptr(), 256, -3.0, 50.0, 1.0, 0.99), j["out"].data_ptr(),
              j["nsamples"].data_ptr()) for j in jobs]

    def separate():
        for h, c, p, o, n in ccams:
            L.vr_render(h, c, p, o, n, s)
    t_sep = _time_ms(torch, separate, max(5, args.steps))
    samples = sum(int(j["nsamples"].sum()) for j in jobs)
    _emit({"workload": "batch_64", "jobs": 64, "samples": samples,
                      "graph_ms": t_graph, "separate_ms": t_sep, "speedup": t_sep / t_graph,
                      "graph_gsamples_per_s": samples / t_graph / 1e6, "separate_gsamples_per_s": samples / t_sep / 1e6,
                      "graph_roofline_frac": gather_rate_frac(samples / t_graph / 1e6, 2),
                      "autotuned": {"brick": brick, "tile": [opts.tile_w, opts.tile_h], "ctas_per_sm": opts.ctas_per_sm,
                                    "warps_per_tile": opts.warps_per_tile}})
    for j in jobs:
        for v in j["vol"].__dict__.get("_rebricked", {}).values():
            v.close()
        j["vol"].close()


def run_diff_512(args):
    """512^3 f32, four 1024^2 views, step 0.5, no early termination: L2 loss
    against targets rendered with a hidden table; forward (one call per view)
    and backward (table and voxel gradients; one call for the four views, and
    one call per view), and their time ratio."""
    import torch
    import paper_1211_4896_gb300 as P
    dev = torch.device("cuda")
    pre = synth.preset_diff_512()
    cube = synth.hi_cube(pre["dims"], pre["n_blobs"], pre["n_disks"], pre["seed"], device=dev)
    vol = P.Volume(cube, "f32")
    hidden = torch.from_numpy(synth.tf_ramp(256)).to(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(5)
    tf = (hidden + 0.05 * torch.rand(hidden.shape, device=dev, generator=gen)).clamp(0, 1).contiguous()
    cams = pre["cameras"]
    tgts = [P.render(vol, c, hidden, synth.TF_VMIN, synth.TF_VMAX, pre["step"], 2.0)[0] for c in cams]
    outs = [torch.empty((1024, 1024, 4), device=dev) for _ in cams]
    nss = [torch.empty((1024, 1024), device=dev, dtype=torch.int32) for _ in cams]
    gtf = torch.empty((256, 4), device=dev, dtype=torch.float64)
    gvox = torch.empty(vol.shape, device=dev)
    grads = [torch.empty_like(o) for o in outs]

    def fwd():
        for c, o, n in zip(cams, outs, nss):
            P.render(vol, c, tf, synth.TF_VMIN, synth.TF_VMAX, pre["step"], 2.0, out=o, nsamples=n)

    def bwd():              # the loss summed over the four views: one multi-view backward call
        for o, g, t in zip(outs, grads, tgts):
            torch.sub(o, t, out=g).mul_(2.0)
        P.render_backward_views(vol, cams, tf, synth.TF_VMIN, synth.TF_VMAX, pre["step"], outs, nss, grads, 2.0,
                                grad_tf=gtf, grad_vox=gvox)

    def bwd_per_view():     # the same as one vr_render_backward call per view
        for v, (c, o, n, g, t) in enumerate(zip(cams, outs, nss, grads, tgts)):
            torch.sub(o, t, out=g).mul_(2.0)
            P.render_backward(vol, c, tf, synth.TF_VMIN, synth.TF_VMAX, pre["step"], o, n, g, 2.0, grad_tf=gtf,
                              grad_vox=gvox, accumulate=v > 0)
    t_f = _time_ms(torch, fwd, max(5, args.steps))
    t_b = _time_ms(torch, bwd, max(5, args.steps))
    t_bv = _time_ms(torch, bwd_per_view, max(5, args.steps))
    samples = sum(int(n.sum()) for n in nss)
    _emit({"workload": "diff_512", "samples": samples, "fwd_ms_4_views": t_f, "bwd_ms_4_views": t_b,
                      "bwd_over_fwd": t_b / t_f, "bwd_ms_per_view_calls": t_bv, "bwd_per_view_calls_over_fwd":
                      t_bv / t_f, "fwd_gsamples_per_s": samples / t_f / 1e6,
                      "fwd_roofline_frac": gather_rate_frac(samples / t_f / 1e6, 4),
                      "fwd_bwd_gsamples_per_s": samples / (t_f + t_b) / 1e6})
    vol.close()


def run_modes_1024(args, mode_name):
    """The 1024^3 float32 cube and the eight 1080p orbit views of the default
    workload, rendered per view (vr_render) with maximum intensity projection
    or the sigma-clipping transfer function (mini-map of 32^3 regions, table
    over [0, 8] sigma); step 1, no early termination for MIP, 0.99 for sigma.
    Pixel error against the oracle on three sampled rows of view 0."""
    import torch
    import oracle
    import paper_1211_4896_gb300 as P
    dev = torch.device("cuda")
    pre = synth.preset_scale_1024()
    cube = make_cube(pre, dev)
    vol = P.Volume(cube, "f32")
    host = cube.cpu().numpy()
    del cube
    torch.cuda.empty_cache()
    tf_np = synth.tf_ramp(256)
    tf = torch.from_numpy(tf_np).to(dev)
    cams = pre["cameras"]
    outs = [torch.empty((1080, 1920, 4), device=dev) for _ in cams]
    nss = [torch.empty((1080, 1920), device=dev, dtype=torch.int32) for _ in cams]
    region = (32, 32, 32)
    res = {"workload": mode_name + "_1024", "views": len(cams), "image": [1920, 1080]}
    if mode_name == "mip":
        kw = dict(mode=P.VR_MODE_MIP)
        vmin, vmax, ert = synth.TF_VMIN, synth.TF_VMAX, 2.0
    else:
        mm = P.minimap(vol, region)
        res["minimap_ms"] = _time_ms(torch, lambda: P.minimap(vol, region, out=mm), 5)
        res["minimap_region"] = list(region)
        kw = dict(mode=P.VR_MODE_SIGMA, minimap=mm, region=region)
        vmin, vmax, ert = 0.0, 8.0, 0.99

    def f():
        for c, o, n in zip(cams, outs, nss):
            P.render(vol, c, tf, vmin, vmax, 1.0, ert, out=o, nsamples=n, **kw)
    ms = _time_ms(torch, f, max(3, args.steps))
    samples = sum(int(n.sum()) for n in nss)
    gs = samples / ms / 1e6
    rows = [440, 540, 640]
    if mode_name == "mip":
        ref = oracle.render_mip(host, cams[0], tf_np, vmin, vmax, 1.0, rows=(rows[0], rows[-1] + 1))
    else:
        stats = oracle.minimap(host, region)
        ref = oracle.render_sigma(host, cams[0], tf_np, vmin, vmax, 1.0, stats, region, ert=ert,
                                  rows=(rows[0], rows[-1] + 1))
    # the sample-count margins of the same rays come from the plain render; these
    # modes report no early-termination margin, so an ERT difference always fails
    plain = oracle.render(host, cams[0], tf_np, synth.TF_VMIN, synth.TF_VMAX, 1.0, 2.0, rows=(rows[0], rows[-1] + 1))
    ref = dict(ref, margin_n=plain["margin_n"], margin_ert=np.full(plain["margin_n"].shape, np.inf))
    res.update({"ms_8_views": ms, "samples": samples, "gsamples_per_s": gs,
                "roofline_frac": gs * 32 / measured_peaks()[0], "roofline_peak_source": measured_peaks()[1],
                "px_err": _px_err(outs[0].cpu().numpy(), nss[0].cpu().numpy(), ref, rows)})
    _emit(res)
    vol.close()


def run_stats_1024(args):
    """Global statistics of the 1024^3 float32 cube (Sections 4.1-4.3):
    moments (one pass), a 256-bin histogram over [min, max] (one pass) and the
    exact median (three passes), each streamed from the bricks; achieved
    bandwidth = bricked bytes read / time, against the measured HBM copy
    bandwidth.  Checked against the oracle."""
    import torch
    import oracle
    import paper_1211_4896_gb300 as P
    dev = torch.device("cuda")
    pre = synth.preset_scale_1024()
    cube = make_cube(pre, dev)
    vol = P.Volume(cube, "f32")
    host = cube.cpu().numpy()
    del cube
    torch.cuda.empty_cache()
    bricked = vol.info["bytes"]
    peak, src = measured_peaks()
    s = int(torch.cuda.current_stream().cuda_stream)
    from paper_1211_4896_gb300 import _lib as L
    mom = torch.empty(5, device=dev, dtype=torch.float64)
    med = torch.empty(1, device=dev, dtype=torch.float64)
    m = P.moments(vol)
    hist = torch.empty(256, device=dev, dtype=torch.int64)
    reps = max(5, args.steps)
    t_m = _time_ms(torch, lambda: L.vr_moments(vol.handle, mom.data_ptr(), s), reps)
    t_h = _time_ms(torch, lambda: L.vr_histogram(vol.handle, m["min"], m["max"], 256, hist.data_ptr(), s), reps)
    t_q = _time_ms(torch, lambda: L.vr_median(vol.handle, med.data_ptr(), s), reps)
    r = oracle.moments(host)
    ok = (m["count"] == r["count"] and abs(m["sd"] - r["sd"]) <= 1e-6 * r["sd"]
          and np.array_equal(hist.cpu().numpy(), oracle.histogram(host, m["min"], m["max"], 256).astype(np.int64))
          and float(med.item()) == oracle.median(host)[0])
    res = {"workload": "stats_1024", "voxels": int(host.size), "bricked_bytes": bricked,
           "moments": {"ms": t_m, "gb_per_s": bricked / t_m / 1e6, "frac": bricked / t_m / 1e6 / peak},
           "histogram_256": {"ms": t_h, "gb_per_s": bricked / t_h / 1e6, "frac": bricked / t_h / 1e6 / peak},
           "median_3_passes": {"ms": t_q, "gb_per_s": 3 * bricked / t_q / 1e6,
                               "frac": 3 * bricked / t_q / 1e6 / peak},
           "peak_gb_per_s": peak, "peak_source": src, "matches_oracle": bool(ok),
           "values": {"mean": m["mean"], "sd": m["sd"], "median": float(med.item())}}
    _emit(res)
    vol.close()


def run_sortlast_1024(args):
    """Sort-last rendering of the 1024^3 float32 cube split into 2x2x2
    sub-boxes of cells (the paper's sub-cubes), eight 1080p orbit views, step 1,
    no early termination: 8 sub-box renders + one depth-ordered composite per
    view, against the whole render of the same views; pixel error of the
    composite against the oracle on three rows of view 0.  The same split
    once more as across GPUs: each box rendered from a volume that holds only
    its sub-cube (vr_render_subbox_of), whose composite must equal the
    whole-volume form bit for bit."""
    import torch
    import oracle
    import paper_1211_4896_gb300 as P
    from paper_1211_4896_gb300.sortlast import sub_cube
    dev = torch.device("cuda")
    pre = synth.preset_scale_1024()
    cube = make_cube(pre, dev)
    vol = P.Volume(cube, "f32")
    e = (0, 511, 1023)                        # 1023 cells per axis, split in two
    boxes = [((e[x], e[y], e[z]), (e[x + 1], e[y + 1], e[z + 1])) for z in (0, 1) for y in (0, 1) for x in (0, 1)]
    sub_vols = [P.Volume(sub_cube(cube, lo, hi), "f32", origin=tuple(float(q) for q in lo)) for lo, hi in boxes]
    dims = tuple(vol.shape[::-1])
    host = cube.cpu().numpy()
    del cube
    torch.cuda.empty_cache()
    tf_np = synth.tf_ramp(256)
    tf = torch.from_numpy(tf_np).to(dev)
    cams = pre["cameras"]
    whole = [torch.empty((1080, 1920, 4), device=dev) for _ in cams]
    nss = [torch.empty((1080, 1920), device=dev, dtype=torch.int32) for _ in cams]
    outs = [torch.empty((1080, 1920, 4), device=dev) for _ in cams]
    from paper_1211_4896_gb300 import _lib as L
    s = int(torch.cuda.current_stream().cuda_stream)
    parts = [[torch.empty((1080, 1920, 4), device=dev) for _ in boxes] for _ in cams]
    depths = [[torch.empty((1080, 1920), device=dev) for _ in boxes] for _ in cams]
    par = L.make_params(tf.data_ptr(), 256, synth.TF_VMIN, synth.TF_VMAX, 1.0, 2.0)

    def f_whole():
        for c, o, n in zip(cams, whole, nss):
            P.render(vol, c, tf, synth.TF_VMIN, synth.TF_VMAX, 1.0, 2.0, out=o, nsamples=n)

    def f_sort_last():
        for v, c in enumerate(cams):
            cc = L.make_camera(c)
            for b, (lo, hi) in enumerate(boxes):
                L.vr_render_subbox(vol.handle, cc, par, lo, hi, parts[v][b].data_ptr(), depths[v][b].data_ptr(),
                                   None, s)
            L.vr_composite([p.data_ptr() for p in parts[v]], [d.data_ptr() for d in depths[v]], 1920, 1080,
                           (0, 0, 0, 0), outs[v].data_ptr(), s)
    outs_sub = [torch.empty((1080, 1920, 4), device=dev) for _ in cams]

    def f_sub_cubes():
        for v, c in enumerate(cams):
            cc = L.make_camera(c)
            for b, (lo, hi) in enumerate(boxes):
                L.vr_render_subbox_of(sub_vols[b].handle, dims, lo, cc, par, lo, hi, parts[v][b].data_ptr(),
                                      depths[v][b].data_ptr(), None, s)
            L.vr_composite([p.data_ptr() for p in parts[v]], [d.data_ptr() for d in depths[v]], 1920, 1080,
                           (0, 0, 0, 0), outs_sub[v].data_ptr(), s)
    reps = max(3, args.steps)
    t_whole = _time_ms(torch, f_whole, reps)
    t_sub = _time_ms(torch, f_sub_cubes, reps)
    t_sl = _time_ms(torch, f_sort_last, reps)
    same = all(torch.equal(a, b) for a, b in zip(outs, outs_sub))
    samples = sum(int(n.sum()) for n in nss)
    rows = [440, 540, 640]
    ref = oracle.render(host, cams[0], tf_np, synth.TF_VMIN, synth.TF_VMAX, 1.0, 2.0, rows=(rows[0], rows[-1] + 1))
    err = _px_err(outs[0].cpu().numpy(), nss[0].cpu().numpy(), ref, rows)
    _emit({"workload": "sortlast_1024", "subboxes": len(boxes), "views": len(cams),
                      "whole_ms_8_views": t_whole, "sort_last_ms_8_views": t_sl, "overhead": t_sl / t_whole,
                      "samples": samples, "sort_last_gsamples_per_s": samples / t_sl / 1e6,
                      "sort_last_roofline_frac": gather_rate_frac(samples / t_sl / 1e6, 4),
                      "max_diff_vs_whole": float(max((o - w).abs().max().item() for o, w in zip(outs, whole))),
                      "sub_cube_volumes_ms_8_views": t_sub, "sub_cube_volumes_bit_identical": same,
                      "px_err": err})
    for sv in sub_vols:
        sv.close()
    vol.close()


def run_skip_1024(args):
    """Exact empty-space skipping on the 1024^3 float32 cube and eight 1080p
    views with a source-finding table (opacity 0 below v = 6, i.e. six noise
    sigmas; most 16^3 bricks hold only noise): the plain march (texture
    layers, and the bricks with them off) and the skipping march (texture
    layers), which must give identical images; rates on nominal samples (those
    marched or skipped up to early termination)."""
    import torch
    import paper_1211_4896_gb300 as P
    dev = torch.device("cuda")
    pre = synth.preset_scale_1024()
    cube = make_cube(pre, dev)
    vol = P.Volume(cube, "f32")
    del cube
    torch.cuda.empty_cache()
    K = 256
    v = synth.TF_VMIN + (synth.TF_VMAX - synth.TF_VMIN) * np.arange(K) / (K - 1)
    t = (v - synth.TF_VMIN) / (synth.TF_VMAX - synth.TF_VMIN)
    a = np.where(v < 6.0, 0.0, 0.02 + 0.2 * (v - 6.0) / (synth.TF_VMAX - 6.0))
    tf = torch.from_numpy(np.stack([t, t * t, 1 - t, a], 1).astype(np.float32)).to(dev)
    cams = pre["cameras"]
    plain = [torch.empty((1080, 1920, 4), device=dev) for _ in cams]
    skip = [torch.empty((1080, 1920, 4), device=dev) for _ in cams]
    nsp = [torch.empty((1080, 1920), device=dev, dtype=torch.int32) for _ in cams]
    nss = [torch.empty((1080, 1920), device=dev, dtype=torch.int32) for _ in cams]

    def run(outs, nss_, flag):
        def f():
            for c, o, n in zip(cams, outs, nss_):
                P.render(vol, c, tf, synth.TF_VMIN, synth.TF_VMAX, 1.0, 0.99, out=o, nsamples=n, skip_empty=flag)
        return f
    reps = max(3, args.steps)
    t_plain = _time_ms(torch, run(plain, nsp, False), reps)
    t_skip = _time_ms(torch, run(skip, nss, True), reps)
    # both marches read texture layers by default; the plain one again on the
    # bricks (layers off) for the rate of the brick layout
    os.environ["VR_TEX_LAYERS"] = "0"
    try:
        t_plain_bricks = _time_ms(torch, run(plain, nsp, False), reps)
    finally:
        del os.environ["VR_TEX_LAYERS"]
    samples = sum(int(n.sum()) for n in nsp)
    same = all(torch.equal(x, y) for x, y in zip(plain, skip)) and all(torch.equal(x, y) for x, y in zip(nsp, nss))
    _emit({"workload": "skip_1024", "views": len(cams), "plain_ms_8_views": t_plain,
                      "plain_bricks_ms_8_views": t_plain_bricks,
                      "skip_ms_8_views": t_skip, "speedup": t_plain / t_skip, "nominal_samples": samples,
                      "plain_gsamples_per_s": samples / t_plain / 1e6, "skip_gsamples_per_s": samples / t_skip / 1e6,
                      "skip_roofline_frac_nominal": gather_rate_frac(samples / t_skip / 1e6, 4),
                      "bit_identical": bool(same)})
    vol.close()


def run_tex_1024(args):
    """The hardware texture filter as a measured alternative (the paper kept
    its sub-cubes in texture memory, Section 4.3): the 1024^3 float32 cube and
    eight 1080p views of the default workload, step 1, ERT 0.99, rendered per
    view with the software trilinear (vr_render) and with the texture unit's
    filter (8 fractional bits of weight).  Rate of each, and the pixel error of
    each against the FP64 oracle on three rows of every view; the texture
    path's error is reported, not held to 1e-4."""
    import torch
    import oracle
    import paper_1211_4896_gb300 as P
    dev = torch.device("cuda")
    pre = synth.preset_scale_1024()
    cube = make_cube(pre, dev)
    vol = P.Volume(cube, "f32")
    host = cube.cpu().numpy()
    del cube
    torch.cuda.empty_cache()
    tf_np = synth.tf_ramp(256)
    tf = torch.from_numpy(tf_np).to(dev)
    cams = pre["cameras"]
    H, W = cams[0]["height"], cams[0]["width"]
    res = {"workload": "tex_1024", "views": len(cams), "image": [W, H]}
    refs = []
    for v, cam in enumerate(cams):
        rows = [H // 2 - 100 + 7 * v, H // 2 + 7 * v, H // 2 + 100 + 7 * v]
        refs.append((rows, _oracle_rows(oracle, host, cam, tf_np, synth.TF_VMIN, synth.TF_VMAX, 1.0, 0.99, rows)))
    for name, flt in (("software", P.VR_FILTER_SOFTWARE), ("texture", P.VR_FILTER_TEXTURE)):
        outs = [torch.empty((H, W, 4), device=dev) for _ in cams]
        nss = [torch.empty((H, W), device=dev, dtype=torch.int32) for _ in cams]

        def f():
            for c, o, n in zip(cams, outs, nss):
                P.render(vol, c, tf, synth.TF_VMIN, synth.TF_VMAX, 1.0, 0.99, filter=flt, out=o, nsamples=n)
        ms = _time_ms(torch, f, max(3, args.steps))
        samples = sum(int(n.sum()) for n in nss)
        errs = [_px_err(o.cpu().numpy(), n.cpu().numpy(), ref, rows, tol=1.0 if flt else PX_TOL_F32)
                for o, n, (rows, ref) in zip(outs, nss, refs)]
        res[name] = {"ms_8_views": ms, "gsamples_per_s": samples / ms / 1e6,
                     "roofline_frac": gather_rate_frac(samples / ms / 1e6, 4),
                     "px_err": _merge_px(errs, "FP64 oracle, three rows of each view")}
    res["texture_over_software_rate"] = res["texture"]["gsamples_per_s"] / res["software"]["gsamples_per_s"]
    _emit(res)
    vol.close()


def run_half_1024(args):
    """The 1024^3 cube and eight 1080p views of the default workload stored
    f32, f16 and bf16: the batched forward of the eight views (one graph call)
    and the eight single-view renders; f32 through the texture layers (its
    default for these dense views) and through the brick copies (layers off),
    so that the 16-bit rates stand against both."""
    import torch
    import paper_1211_4896_gb300 as P
    from paper_1211_4896_gb300 import _lib as L
    dev = torch.device("cuda")
    pre = synth.preset_scale_1024()
    cube = make_cube(pre, dev)
    tf = torch.from_numpy(synth.tf_ramp(256)).to(dev)
    cams = pre["cameras"]
    s_ptr = int(torch.cuda.current_stream().cuda_stream)
    res = {"workload": "half_1024", "views": len(cams), "image": [1920, 1080]}
    ref = None
    for store, layers in (("f32", True), ("f32", False), ("f16", False), ("bf16", False)):
        if not layers:
            os.environ["VR_TEX_LAYERS"] = "0"
        try:
            vol = P.Volume(cube, store)
            outs = [torch.empty((1080, 1920, 4), device=dev) for _ in cams]
            nss = [torch.empty((1080, 1920), device=dev, dtype=torch.int32) for _ in cams]
            jobs = [dict(vol=vol, cam=c, tf=tf, vmin=synth.TF_VMIN, vmax=synth.TF_VMAX, step=1.0, ert=0.99, out=o,
                         nsamples=n) for c, o, n in zip(cams, outs, nss)]
            cj = P.render_batched(jobs, use_graph=True)
            opts = L.vr_batch_opts(1, 8, 4, 0)
            t_bat = _time_ms(torch, lambda: L.vr_render_batched(cj, opts, s_ptr), max(5, args.steps))
            ccams = [L.make_camera(c) for c in cams]
            cpar = L.make_params(tf.data_ptr(), 256, synth.TF_VMIN, synth.TF_VMAX, 1.0, 0.99)

            def single():
                for cc, o, n in zip(ccams, outs, nss):
                    L.vr_render(vol.handle, cc, cpar, o.data_ptr(), n.data_ptr(), s_ptr)
            t_one = _time_ms(torch, single, max(5, args.steps))
            samples = sum(int(n.sum()) for n in nss)
            key = store + ("_layers" if layers else "_bricks")
            r = {"batched_ms_8_views": t_bat, "batched_gsamples_per_s": samples / t_bat / 1e6,
                 "single_ms_8_views": t_one, "single_gsamples_per_s": samples / t_one / 1e6,
                 "layouts": sorted({L.vr_view_layout(vol.handle, cc) for cc in ccams})}
            if ref is None:
                ref = [o.clone() for o in outs]
            else:
                r["max_abs_diff_vs_f32"] = max(float((o - q).abs().max()) for o, q in zip(outs, ref))
            res[key] = r
            vol.close()
            torch.cuda.empty_cache()
        finally:
            os.environ.pop("VR_TEX_LAYERS", None)
    for st in ("f16", "bf16"):
        for base in ("f32_layers", "f32_bricks"):
            res["%s_over_%s_batched" % (st, base)] = res[base]["batched_ms_8_views"] / res[st + "_bricks"]["batched_ms_8_views"]
    _emit(res)


def _oracle_rate(fn, cores, min_s=1.0):
    """Composited samples per second of fn(nthreads) -> samples, repeated
    until min_s seconds have passed (one call at least)."""
    t0 = time.perf_counter()
    samples, calls = 0, 0
    while True:
        samples += fn(cores)
        calls += 1
        t = time.perf_counter() - t0
        if t >= min_s:
            break
    return {"cores": cores, "calls": calls, "seconds": t, "samples": samples, "gsamples_per_s": samples / t / 1e9}


def run_cpu_oracle(args):
    """The FP64 oracle timed on the host cores, with every core and with one,
    on the paper-scale workloads (CPU only; the cubes are generated on the GPU
    when there is one, outside the timed calls):
      plain_128   the whole 256^2 render of the 128^3 cube (forward);
      scale_1024  one full 1080p view (view 0) of the 1024^3 cube, forward +
                  backward (table gradient), as in the headline's cpu_baseline;
      precision   one full 1080p view of the 256^3 crop of the 4096^2 x 1024
                  cube that the precision workload checks pixels on (forward);
      diff_crop   the 32^3 crop (around the brightest voxel) of the 512^3
                  differentiation cube, its four 64^2 views: forward + backward
                  with table and voxel gradients."""
    import torch
    import oracle
    dev = torch.device("cuda") if torch.cuda.is_available() else torch.device("cpu")
    ncores = os.cpu_count() or 1
    tf_np = synth.tf_ramp(256)
    vmin, vmax = synth.TF_VMIN, synth.TF_VMAX
    out = {"workload": "cpu_oracle", "host_cores": ncores, "machine": platform.machine(), "rows": {}}

    def both(name, fn, desc, min_s):
        out["rows"][name] = {"what": desc, "all_cores": _oracle_rate(fn, ncores, min_s),
                             "one_core": _oracle_rate(fn, 1, min_s)}
        print("cpu_oracle: %s done" % name, file=sys.stderr)

    # plain_128
    pre = synth.preset_plain_128()
    host = synth.hi_cube(pre["dims"], pre["n_blobs"], pre["n_disks"], pre["seed"]).numpy()
    cam = pre["cameras"][0]
    both("plain_128", lambda nt: int(oracle.render(host, cam, tf_np, vmin, vmax, pre["step"], pre["ert"],
                                                   nthreads=nt)["n_used"].sum()),
         "128^3 f32, orthographic 256^2 along +z, step 0.5, no ERT; whole image, forward", 2.0)
    # scale_1024, one full view
    pre = synth.preset_scale_1024()
    host = make_cube(pre, dev).cpu().numpy()
    torch.cuda.empty_cache() if dev.type == "cuda" else None
    cam = pre["cameras"][0]
    g = np.random.default_rng(0).normal(size=(cam["height"], cam["width"], 4))

    def c2(nt):
        o = oracle.render(host, cam, tf_np, vmin, vmax, pre["step"], pre["ert"], nthreads=nt)
        oracle.render_backward(host, cam, tf_np, vmin, vmax, pre["step"], g, ert=pre["ert"], want_vox=False,
                               nthreads=nt)
        return int(o["n_used"].sum())
    both("scale_1024", c2, "1024^3 f32, view 0 of the 8 orbit views (1920x1080), step 1, ERT 0.99; forward + "
                           "backward (table gradient)", 0.0)
    del host
    # precision crop
    dims = (4096, 4096, 1024)
    nb = int(round(20 * (4096 * 4096 * 1024) / 128 ** 3))
    nd = int(round(200 * (4096 * 4096 * 1024) / 1024 ** 3))
    cube = synth.hi_cube(dims, nb, nd, seed=3, device=dev)
    crop = cube[384:640, 1920:2176, 1920:2176].contiguous().cpu().numpy()
    del cube
    torch.cuda.empty_cache() if dev.type == "cuda" else None
    cam = synth.orbit_cameras((256, 256, 256), 4, 40.0, 1920, 1080, start_deg=30.0)[0]
    both("precision_crop", lambda nt: int(oracle.render(crop, cam, tf_np, vmin, vmax, 1.0, 0.99,
                                                        nthreads=nt)["n_used"].sum()),
         "the 256^3 f32 crop of the 4096^2 x 1024 cube, its first 1920x1080 orbit view, step 1, ERT 0.99; forward",
         0.0)
    # differentiation crop
    pre = synth.preset_diff_512()
    cube = synth.hi_cube(pre["dims"], pre["n_blobs"], pre["n_disks"], pre["seed"], device=dev)
    n = 32
    centre = np.unravel_index(int(torch.argmax(cube).item()), cube.shape)
    lo = [int(min(max(c - n // 2, 0), d - n)) for c, d in zip(centre, cube.shape)]
    crop = cube[lo[0]:lo[0] + n, lo[1]:lo[1] + n, lo[2]:lo[2] + n].contiguous().cpu().numpy()
    del cube
    cams = synth.orbit_cameras((n, n, n), 4, 40.0, 64, 64, start_deg=20.0)
    gr = [np.random.default_rng(10 + q).normal(size=(64, 64, 4)) for q in range(4)]

    def c5(nt):
        s = 0
        for c, gq in zip(cams, gr):
            s += int(oracle.render(crop, c, tf_np, vmin, vmax, pre["step"], 2.0, nthreads=nt)["n_used"].sum())
            oracle.render_backward(crop, c, tf_np, vmin, vmax, pre["step"], gq, nthreads=nt)
        return s
    both("diff_crop", c5, "32^3 f32 crop of the 512^3 differentiation cube, four 64^2 orbit views, step 0.5, "
                          "no ERT; forward + backward (table and voxel gradients)", 2.0)
    out["note"] = ("FP64 oracle (oracle/vr_oracle.c) as it stands, pixels dealt round-robin to pthreads; one_core = one "
                   "thread; each figure repeats its call until at least the given time has passed")
    print(json.dumps(out))


WORKLOADS = {"plain_128": run_plain_128, "precision_4096": run_precision_4096, "batch_64": run_batch_64,
             "diff_512": run_diff_512, "mip_1024": lambda a: run_modes_1024(a, "mip"),
             "sigma_1024": lambda a: run_modes_1024(a, "sigma"), "stats_1024": run_stats_1024,
             "sortlast_1024": run_sortlast_1024, "skip_1024": run_skip_1024, "tex_1024": run_tex_1024,
             "cpu_oracle": run_cpu_oracle, "half_1024": run_half_1024}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="scale_1024", choices=["scale_1024"] + sorted(WORKLOADS))
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank)
    from paper_1211_4896_gb300 import build as B
    B.build()
    if args.workload != "scale_1024":
        import oracle
        oracle.build()
        return WORKLOADS[args.workload](args) or 0
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
