"""Benchmark: one step = zero accumulator -> simulate the paper-scale
workload's histories -> finalize (3D Gaussian smoothing sigma = 2 bins,
per-LOR sensitivity multiply) through the C ABI.

Workload (paper scale): 128x128x89 torso phantom (2.34x2.34x2.78 mm, lungs,
spine, 6 hot spheres 4:1), 448-crystal x 45-ring scanner (R 311.8 mm, 250.4
mm), 27 TOF bins with 400 ps FWHM blur, FP32 LUT 64x32x32x16x9, 1e9
histories per step.  Metric: photon-pair histories per second (whole job).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--histories H]
  python bench.py --impl reference ...   (the FP64 CPU oracle on a bounded sample)
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "photon histories/s"
UNIT = "histories/s"
WORKLOAD = "paper-scale torso 128x128x89, scanner 448x45, 27 TOF (400 ps), LUT 64x32x32x16x9 f32, 1e9 histories/step, smoothing sigma=2, per-LOR sensitivity"
WORKLOAD_SMALL = ("small: water cylinder r=100 mm in 64x64x32 voxels of 4 mm, scanner 288x16, 13 TOF bins of 50 mm, "
                  "LUT 16x8x8x4x4 f32, smoothing sigma=2, per-LOR sensitivity")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--histories", type=float, default=1e9)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--mode", default="step",
                    choices=["step", "precision", "accuracy", "batched", "served", "postproc"],
                    help="step: the benchmark line; precision: LUT precision / count-level study; "
                         "batched / served: request server vs plain sequential requests")
    ap.add_argument("--requests", type=int, default=32, help="batched: phantoms; served: chains")
    ap.add_argument("--rate", type=float, default=20.0, help="served: mean request arrivals per s")
    ap.add_argument("--max-active", type=int, default=4)
    ap.add_argument("--budget-scale", type=float, default=1.0,
                    help="multiply the 1e6-1e9 history budgets (shorter runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-requests", action="store_true",
                    help="step mode: skip the batched / served request mixes after the timed steps")
    ap.add_argument("--served-chains", type=int, default=12,
                    help="step mode: chains of the served request mix")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rings", type=int, default=0,
                    help="profiling case: keep only this many rings (smaller sinogram)")
    ap.add_argument("--tof-bins", type=int, default=0,
                    help="profiling case: this many TOF bins over the same 648 mm range")
    ap.add_argument("--workload", default="paper", choices=["paper", "small"],
                    help="step workload: the paper-scale configuration or the small one")
    ap.add_argument("--e-res", type=float, default=0.0,
                    help="energy resolution FWHM at 511 keV (fraction); the no-LUT mode uses 0.112 "
                         "with the small configuration's 425-650 keV window")
    ap.add_argument("--lut-axes", default="full", choices=["full", "e", "eab", "etz"],
                    help="LUT axes kept (Sec. 2.2.2's lower-dimensional LUTs, from synthetic histograms): "
                         "e energy, ab incidence angles, tz crystal positions")
    ap.add_argument("--gaps", type=int, default=0, choices=[0, 1, 2],
                    help="gaps between modules and blocks: 1 loses photons in a gap, 2 assigns them "
                         "to edge crystals (paper-scale workload; 2 mm gaps, 18 x 55 LUT positions)")
    ap.add_argument("--sigma", type=float, nargs=3, default=[2.0, 2.0, 2.0],
                    help="precision study: smoothing sigma in bins (radial, view, axial); the paper's "
                         "kernel widths, FWHM 10 / 5 / 18 bins, are 4.25 2.12 7.64")
    ap.add_argument("--reference-histories", type=float, default=1e10,
                    help="precision study: histories of the FP32 reference estimate")
    ap.add_argument("--precision-workload", default="small", choices=["small", "paper"],
                    help="precision study on the small configuration (water cylinder, 288 x 16 "
                         "scanner) or the paper-scale one")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    """SM clock and clock-event reasons sampled every 0.2 s while the timed
    region runs.  NVML is read in-process through ctypes (the call releases
    the GIL and forks nothing); without NVML, nvidia-smi is run instead."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits, in the order of the columns above
    BITS = (0x8, 0x40, 0x20, 0x4)

    def __init__(self, device_index):
        self.idx = device_index
        self.samples = []
        self.stop = threading.Event()
        self.t = None
        self.nvml = self._nvml_handle(device_index)
        self.source = "nvml" if self.nvml else "nvidia-smi"

    @staticmethod
    def _nvml_handle(idx):
        import ctypes as C
        try:
            lib = C.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            h = C.c_void_p()
            try:
                import torch
                p = torch.cuda.get_device_properties(idx)
                bus = f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0".encode()
                if lib.nvmlDeviceGetHandleByPciBusId_v2(C.c_char_p(bus), C.byref(h)) != 0:
                    raise OSError
            except Exception:
                if lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(idx), C.byref(h)) != 0:
                    return None
            return lib, h
        except (OSError, AttributeError):
            return None

    def _sample_nvml(self):
        import ctypes as C
        lib, h = self.nvml
        sm, mx, why = C.c_uint(), C.c_uint(), C.c_ulonglong()
        if lib.nvmlDeviceGetClockInfo(h, 1, C.byref(sm)) != 0:  # 1 = NVML_CLOCK_SM
            return
        lib.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(mx))
        try:
            reasons = lib.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            reasons = lib.nvmlDeviceGetCurrentClocksThrottleReasons
        reasons(h, C.byref(why))
        self.samples.append([str(sm.value), str(mx.value)] +
                            ["Active" if why.value & b else "Not Active" for b in self.BITS])

    def _run(self):
        while not self.stop.is_set():
            try:
                if self.nvml:
                    self._sample_nvml()
                else:
                    out = subprocess.check_output(
                        ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                         "--format=csv,noheader,nounits"], text=True, timeout=5)
                    self.samples.append([x.strip() for x in out.strip().split(",")])
            except Exception:
                pass
            self.stop.wait(0.2)

    def __enter__(self):
        self.t = threading.Thread(target=self._run, daemon=True)
        self.t.start()
        return self

    def __exit__(self, *a):
        self.stop.set()
        self.t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > i + 2 and s[i + 2].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples), "source": self.source}


def huge_page_gb(ptr):
    """GB of the mapping holding host address ptr that are backed by
    transparent huge pages (/proc/self/smaps), or None where unreadable."""
    try:
        inside = False
        with open("/proc/self/smaps") as f:
            for line in f:
                head = line.split()[0] if line.strip() else ""
                if "-" in head and all(c in "0123456789abcdef-" for c in head):
                    lo, hi = (int(x, 16) for x in head.split("-"))
                    inside = lo <= ptr < hi
                elif inside and line.startswith("AnonHugePages:"):
                    return round(int(line.split()[1]) * 1024 / 1e9, 2)
    except OSError:
        pass
    return None


def host_memory_state():
    """Host memory facts that bear on device-to-host copies: the cgroup's
    limit and use, this process's resident set, and the kernel's compaction,
    THP and reclaim counters (to difference across the end-to-end leg)."""
    out = {}
    for k, path in (("cgroup_max_gb", "/sys/fs/cgroup/memory.max"), ("cgroup_current_gb", "/sys/fs/cgroup/memory.current")):
        try:
            v = open(path).read().strip()
            out[k] = None if v == "max" else round(int(v) / 1e9, 2)
        except (OSError, ValueError):
            pass
    try:
        for line in open("/proc/self/status"):
            if line.startswith("VmRSS:"):
                out["rss_gb"] = round(int(line.split()[1]) * 1024 / 1e9, 2)
    except OSError:
        pass
    keys = ("compact_stall", "compact_fail", "thp_fault_alloc", "thp_fault_fallback", "thp_collapse_alloc",
            "thp_split_page", "thp_split_pmd", "thp_underused_split_page", "thp_deferred_split_page",
            "thp_migration_split", "thp_migration_fail", "pgmigrate_success",
            "pgmigrate_fail", "pgscan_direct", "pgsteal_direct", "pgmajfault")
    try:
        for line in open("/proc/meminfo"):
            name, val = line.split(":", 1)
            if name in ("CmaTotal", "CmaFree", "MemFree", "AnonHugePages"):
                out[name] = round(int(val.split()[0]) * 1024 / 1e9, 2)
    except (OSError, ValueError):
        pass
    try:
        vm = dict(line.split() for line in open("/proc/vmstat"))
        out["vmstat"] = {k: int(vm[k]) for k in keys if k in vm}
    except (OSError, ValueError):
        pass
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# algorithmic work of the transport kernel (lane operations), per counter:
# fixed per-operation costs written from the algorithm (a Philox block is 10
# rounds of 2 wide multiplies, 4 XORs and 2 key adds), not from the code
# ---------------------------------------------------------------------------
OPS_PER_PHILOX_BLOCK = 100
OPS_PER_STEP = 40
OPS_PER_TRY = 15
OPS_PER_INTERACTION = 45
OPS_PER_DETECTION = 110
OPS_PER_HISTORY = 60
# DRAM bytes (read + write) per history of the transport kernel, from an ncu
# capture of the same kernel on the paper-scale torso with the TOF axis
# folded to one bin (the full 43.8 GB accumulator is too large to capture);
# the traffic is the binned atomics and LUT misses, so it scales with the
# histories of a launch
TRANSPORT_DRAM_BYTES_PER_HISTORY = (113.73e6 + 24.62e6) / 2e7  # ncu dram bytes of one 2e7-history launch (profiles/)
# HBM bytes per bin of the smoothing finalize.  The method's own: the int64
# accumulator read once and the FP64 estimate written once, plus the per-LOR
# FP64 sensitivity (8 / n_tof per bin).  The three-pass design moves two FP32
# intermediates on top: radial 8 + 4, view 4 + 4, axial 4 + 8 = 32.
FINALIZE_METHOD_BYTES_PER_BIN = 16
FINALIZE_DESIGN_BYTES_PER_BIN = 32
# DRAM bytes (read + write) per bin of the smoothing launches of one
# finalize, from an ncu capture of the paper-scale scanner cut to 5 rings (27
# TOF bins, 67.6 M bins; profiles/finalize_traffic_5_rings_27tof.md): the
# traffic grows with the bins, so it scales to the full sinogram
FINALIZE_DRAM_BYTES_PER_BIN = (1109.3e6 + 884.0e6) / 67_586_400


def transport_ops(st):
    det = st["detected"]
    hist = sum(st[c] for c in ("absorbed", "lost_axial", "energy_window", "step_limit",
                                "same_crystal", "out_of_range", "true", "scatter"))
    return (OPS_PER_PHILOX_BLOCK * st["rng_blocks"] + OPS_PER_STEP * st["steps"]
            + OPS_PER_TRY * st["tries"] + OPS_PER_INTERACTION * (st["compton"] + st["rayleigh"])
            + OPS_PER_DETECTION * det + OPS_PER_HISTORY * hist)


def transport_bounds(psc, st, kern_ms, big, stream):
    """The transport's random-access rates against what the device sustains:
    int64 atomic adds spread over a sinogram-sized buffer (the output buffer,
    viewed as int64, stands in for the accumulator) and 4-byte gathers from a
    64 MB table (the size of the phantom, alias table and LUT together).  The
    transport's rates come from its device counters over the mean timed
    launch: one atomic per bin a warp adds to, an alias entry per history, a
    material and a density per Woodcock step, and 8 LUT taps per photon of a
    binned coincidence."""
    import torch
    sh = stream.cuda_stream
    buf = big.view(torch.int64).view(-1)
    table = torch.rand(16 << 20, device=big.device)
    sink = torch.zeros(1, device=big.device)
    grid, block = 152 * 8, 256

    def timed(fn, per_thread, reps=3):
        fn(per_thread)                                   # warm-up
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(per_thread)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        return grid * block * per_thread / best

    atom_peak = timed(lambda k: psc.psc_peak_random_atomics(buf, grid, block, k, seed=7, stream=sh), 256)
    gath_peak = timed(lambda k: psc.psc_peak_random_gather(table, sink, grid, block, k, seed=7, stream=sh), 512)
    del table
    hist = sum(st[c] for c in ("absorbed", "lost_axial", "energy_window", "step_limit",
                                "same_crystal", "out_of_range", "true", "scatter"))
    kern_s = kern_ms / 1e3
    atom = st["atomics"] / kern_s
    gath = (hist + 2 * st["steps"] + 16 * st["binned"]) / kern_s
    return {"atomics": {"achieved": round(atom / 1e9, 4), "peak": round(atom_peak / 1e9, 3), "unit": "G/s",
                        "frac": round(atom / atom_peak, 4),
                        "peak_source": "random int64 atomicAdd over a 43.8 GB buffer (psc_peak_random_atomics)"},
            "l2_gathers": {"achieved": round(gath / 1e9, 3), "peak": round(gath_peak / 1e9, 2), "unit": "G/s",
                           "frac": round(gath / gath_peak, 4),
                           "peak_source": "random 4-byte loads from a 64 MB table (psc_peak_random_gather)"}}


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------
def build_inputs(rings=0, tof_bins=0, workload="paper", gaps=0):
    if workload == "small":
        sc = W.scanner_tiny()
        return (sc, W.standard_materials(), W.phantom_water_cylinder(), W.lut_tiny(sc),
                W.sensitivity_uniform(sc.lor_shape, seed=1))
    sc = W.scanner_signa()
    if rings:
        sc = W.Scanner(sc.radius, sc.n_crystals, rings, sc.ring_pitch, sc.module_t, sc.module_a,
                       sc.e_lo, sc.e_hi, sc.n_tof, sc.tof_bin_mm, sc.tof_sigma_mm)
    if tof_bins:
        sc.tof_bin_mm = sc.n_tof * sc.tof_bin_mm / tof_bins
        sc.n_tof = tof_bins
    if gaps:
        g = W.scanner_signa_gaps(gap_mode=gaps)
        sc.gap_mode, sc.gap_t, sc.gap_a = g.gap_mode, g.gap_t, g.gap_a
    mats = W.standard_materials()
    ph = W.phantom_torso()
    lut = W.lut_signa(sc)
    sens = W.sensitivity_uniform(sc.lor_shape, seed=1)
    return sc, mats, ph, lut, sens


def workload_inputs(a):
    """The step workload the options name: inputs and its description."""
    if a.gaps and a.workload != "paper":
        raise SystemExit("--gaps applies to the paper-scale workload")
    sc, mats, ph, lut, sens = build_inputs(a.rings, a.tof_bins, a.workload, a.gaps)
    if a.e_res > 0:
        sc.e_res = a.e_res
    keep = {"e": ("e",), "eab": ("e", "a", "b"), "etz": ("e", "t", "z")}.get(a.lut_axes)
    if keep is not None:
        inc, det = W.lut_histograms(lut, counts=50.0)
        lut = W.lut_reduced(lut, inc, det, keep)
    base_wl = WORKLOAD_SMALL if a.workload == "small" else WORKLOAD
    workload = base_wl if not (a.rings or a.tof_bins) else \
        f"profiling case: {base_wl} with {sc.n_rings} rings and {sc.n_tof} TOF bins"
    if a.e_res > 0:
        workload += f", energy resolution {100 * a.e_res:.1f} % FWHM at 511 keV"
    if keep is not None:
        workload += (f", lower-dimensional LUT {lut.n_e}x{lut.n_a}x{lut.n_b}x{lut.n_tpos}x{lut.n_apos} "
                     f"(axes kept: {'+'.join(keep)})")
    if a.gaps:
        workload += (f", {sc.gap_t:g} mm module and {sc.gap_a:g} mm block gaps with LUT positions "
                     f"{sc.n_tpos}x{sc.n_apos}, "
                     + ("photons in a gap lost" if a.gaps == 1 else "edge-crystal assignment"))
    return sc, mats, ph, lut, sens, workload


def step_config(sc, workload, n, world):
    """The config of the step line (both arms)."""
    return {"workload": workload, "histories_per_step": n, "global_batch": world * n,
            "l2": f"inputs larger than L2 ({sc.n_bins * 8 / 1e9:.1f} GB accumulator + "
                  f"{sc.n_bins * 8 / 1e9:.1f} GB output streamed every step)",
            "parallelism": f"replicas{world}"}


def run_native(a):
    import torch
    import torch.distributed as dist
    import paper_2509_05047_gb300 as psc
    from paper_2509_05047_gb300 import build as B
    B.build()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    sc, mats, ph, lut, sens, workload = workload_inputs(a)
    n = int(a.histories)
    ctx = psc.psc_create(local)
    s_id = psc.psc_load_scanner(ctx, psc.scanner_desc(sc))
    m_id = psc.psc_load_materials(ctx, psc.materials_desc(mats).desc)
    p_id = psc.psc_load_phantom(ctx, psc.phantom_desc(ph).desc, m_id)
    l_id = psc.psc_load_lut(ctx, psc.lut_desc(lut).desc)
    sn_id = psc.psc_load_sinogram(ctx, s_id, sens, per_lor=True)
    a_id = psc.psc_acc_create(ctx, s_id)
    out = torch.empty(sc.shape, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    seed = 20250905 + 7919 * rank           # each rank: its own independent request
    fin = psc.finalize_args(a_id, sens=sn_id, sigma=(2.0, 2.0, 2.0), scale=1.0 / n)

    def step(i, ev=None, dst=None):
        if ev is not None:
            ev[0].record(stream)
        psc.psc_acc_zero(ctx, a_id, sh)
        if ev is not None:
            ev[1].record(stream)
        psc.psc_simulate(ctx, psc.sim_args(seed, i * n, n, s_id, p_id, a_id, lut=l_id), stream=sh)
        if ev is not None:
            ev[2].record(stream)
        psc.psc_finalize(ctx, fin, out if dst is None else dst, sh)
        if ev is not None:
            ev[3].record(stream)

    # counters of one step's transport (for the algorithmic-work roofline)
    psc.psc_acc_zero(ctx, a_id, sh)
    st = psc.psc_simulate(ctx, psc.sim_args(seed, 0, n, s_id, p_id, a_id, lut=l_id), stats=True,
                          stream=sh)
    for i in range(a.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(4)) for _ in range(a.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0.record(stream)
        for i in range(a.steps):
            step(a.warmup + i, evs[i])
        t1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = t0.elapsed_time(t1)
    phase = np.array([[e[j].elapsed_time(e[j + 1]) for j in range(3)] for e in evs]).mean(axis=0)
    kern_ms = float(phase[1])
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / a.steps
    value = world * n * a.steps / (ms / 1e3)
    bounds = transport_bounds(psc, st, kern_ms, out, stream) if rank == 0 else None

    # end to end through the C ABI with host buffers: every step a new
    # activity image goes in from the host (psc_update_activity) and the
    # scatter estimate comes back to page-locked host memory
    # (psc_finalize_host into a psc_host_alloc buffer: each finished group of
    # ring-difference segments is copied while the rest is still smoothed).
    # Steps are pipelined the way a caller would run them: the read-back of
    # step i (on a copy stream) overlaps step i+1, with two device work
    # buffers taking turns.  Like the device-timed steps, untimed warm-up
    # steps (with their read-backs) come first, at least W and more while the
    # read-back still speeds up.
    e2e = None
    if not a.no_e2e and rank == 0:
        mem_before = host_memory_state()
        host_out = psc.host_tensor(sc.shape, torch.float64)   # page-locked, huge pages
        mem_alloc = dict(host_memory_state(), buffer_huge_page_gb=huge_page_gb(host_out.data_ptr()))
        act = np.ascontiguousarray(ph.activity, dtype=np.float32)
        outs = [out, torch.empty_like(out)]
        copy = torch.cuda.Stream(dev)

        def e2e_run(i0, k):
            # per step: compute start / transport end / finalize end on the step
            # stream, and the end of the step's copies on the copy stream
            ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(k)]
            torch.cuda.synchronize()
            t_start = time.perf_counter()
            for i in range(k):
                b = i % 2
                psc.psc_update_activity(ctx, p_id, act)   # waits only for launches reading the phantom
                if i >= 2:
                    stream.wait_event(ev[i - 2][3])        # the buffer's previous read-back is done
                ev[i][0].record(stream)
                psc.psc_acc_zero(ctx, a_id, sh)
                psc.psc_simulate(ctx, psc.sim_args(seed, (i0 + i) * n, n, s_id, p_id, a_id, lut=l_id),
                                 stream=sh)
                ev[i][1].record(stream)
                psc.psc_finalize_host(ctx, fin, outs[b], host_out, sh, copy.cuda_stream)
                ev[i][2].record(stream)
                ev[i][3].record(copy)
            torch.cuda.synchronize()
            return time.perf_counter() - t_start, ev

        # warm-up: at least W steps, then more (up to 12 in all) while the read-back is
        # still getting faster by more than 5 % a step
        n_warm, prev = 0, None
        while True:
            _, wev = e2e_run(100 + n_warm, 1)
            n_warm += 1
            back = wev[0][1].elapsed_time(wev[0][3])
            if n_warm >= max(1, a.warmup) and (n_warm >= 12 or (prev is not None and back > 0.95 * prev)):
                break
            prev = back
        k = max(2, a.steps)
        dt, ev = e2e_run(200, k)
        # the copy stream's busy time per step: from the later of the step's
        # finalize start and the previous step's last copy, to its own last copy
        busy = []
        for i in range(k):
            t0i = ev[i][1] if i == 0 else (ev[i][1] if ev[i - 1][3].elapsed_time(ev[i][1]) > 0 else ev[i - 1][3])
            busy.append(t0i.elapsed_time(ev[i][3]))
        nbytes = int(out.numel() * 8)
        e2e = {"value": n * k / dt, "unit": UNIT, "h2d_bytes_per_step": int(act.nbytes),
               "host_buffer_huge_page_gb": huge_page_gb(host_out.data_ptr()),
               "host_memory": {"before": mem_before, "after_alloc": mem_alloc, "after": host_memory_state()},
               "d2h_bytes_per_step": nbytes, "steps": k, "warmup": n_warm,
               "api": "psc_update_activity + psc_acc_zero + psc_simulate + psc_finalize_host (C ABI)",
               "pipelined": "read-back of step i overlaps the smoothing of step i and step i+1 "
                            "(two device work buffers)",
               "ranks_measured": 1,  # rank 0 alone: N ranks' 43.8 GB host buffers do not fit host memory
               "compute_ms": [round(ev[i][0].elapsed_time(ev[i][2]), 1) for i in range(k)],
               "readback_busy_ms": [round(x, 1) for x in busy],
               "readback_gbs": round(nbytes * k / sum(busy) / 1e6, 1)}
        del host_out, outs

    peaks, src = measured_peaks()
    clocks = clk.summary()
    sm_mhz = clocks["sm_mhz"] or peaks.get("clocks_under_load", {}).get("sm_mhz_median", 1485.0)
    peak_ops = 152 * 128 * sm_mhz * 1e6                 # FP32/INT32 lane-ops per second
    ops = transport_ops(st)
    achieved = ops / (kern_ms / 1e3)
    roofline = {"bound": "alu", "achieved": round(achieved / 1e9, 1), "peak": round(peak_ops / 1e9, 1),
                "unit": "Gop/s", "frac": round(achieved / peak_ops, 4),
                "traffic": int(TRANSPORT_DRAM_BYTES_PER_HISTORY * n),
                "kernel": "psc::transport_kernel<0, false, true, true>", "kernel_ms": round(kern_ms, 3),
                "peak_source": f"152 SMs x 128 lanes x median SM clock under load ({sm_mhz:.0f} MHz)"}
    # the three smoothing passes together, against the measured copy bandwidth:
    # achieved on the method's bytes, and the design's own traffic beside it
    method_b = FINALIZE_METHOD_BYTES_PER_BIN + 8.0 / sc.n_tof
    fin_gbs = method_b * sc.n_bins / (phase[2] / 1e3) / 1e9
    design_gbs = (FINALIZE_DESIGN_BYTES_PER_BIN + 8.0 / sc.n_tof) * sc.n_bins / (phase[2] / 1e3) / 1e9
    finalize_roofline = {"bound": "hbm", "achieved": round(fin_gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": round(fin_gbs / peaks["hbm_gbs"], 4),
                         "traffic": round(FINALIZE_DRAM_BYTES_PER_BIN * sc.n_bins),
                         "bytes_per_bin": round(method_b, 3),
                         "design_bytes_per_bin": round(FINALIZE_DESIGN_BYTES_PER_BIN + 8.0 / sc.n_tof, 3),
                         "design_frac": round(design_gbs / peaks["hbm_gbs"], 4),
                         "kernels": "psc::smooth_radial_kernel, psc::smooth_view_kernel, psc::smooth_axial_tma_kernel",
                         "ms": round(float(phase[2]), 3),
                         "peak_source": f"{src} copy bandwidth"}
    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": step_config(sc, workload, n, world),
           "roofline": roofline, "finalize_roofline": finalize_roofline, "transport_bounds": bounds,
           "clocks": clocks, "e2e": e2e,
           "gpu_launches": 4 * a.steps,
           "phases_ms": {"acc_zero": round(float(phase[0]), 3), "transport": round(float(phase[1]), 3),
                         "finalize": round(float(phase[2]), 3)},
           "transport_stats": {k: int(v) for k, v in st.items()}}
    if rank == 0 and not a.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(sc, mats, ph, lut, sens, n, budget_s=20.0)
    psc.psc_destroy(ctx)
    if rank == 0 and world == 1 and not a.no_requests:
        # the request mixes of the batched and served configurations, plain
        # sequential requests against the request server (outside the timed steps)
        del out
        torch.cuda.empty_cache()
        res["requests"] = {
            "batched": run_requests(a, served=False, chains=32, max_active=8),
            "served": run_requests(a, served=True, chains=a.served_chains, max_active=a.max_active)}
        res["config"]["requests"] = (f"batched: 32 seeded torsos 96^3-class to 192x192x120 on the small "
                                     f"scanner, budgets log-uniform 1e6-1e9 x {a.budget_scale:g}, all at t=0; "
                                     f"served: {a.served_chains} chains x 5 iterations (small / paper-scale / "
                                     f"torso), Poisson arrivals {a.rate:g}/s")
    if world > 1:
        dist.destroy_process_group()
    return res if rank == 0 else None


# ---------------------------------------------------------------------------
# oracle on the host cores (bounded sample, extrapolated to one step)
# ---------------------------------------------------------------------------
def cpu_baseline(sc, mats, ph, lut, sens, n, budget_s=20.0):
    import oracle
    cores = os.cpu_count() or 1
    alias = oracle.alias_build(ph.activity)
    m = 20_000
    t = time.perf_counter()
    oracle.simulate(sc, mats, ph, lut, 1, 0, m, threads=cores, alias=alias)
    per_h = (time.perf_counter() - t) / m
    m = int(max(20_000, min(2_000_000, 0.6 * budget_s / max(per_h, 1e-9))))
    t = time.perf_counter()
    oracle.simulate(sc, mats, ph, lut, 2, 0, m, threads=cores, alias=alias)
    per_h = (time.perf_counter() - t) / m
    # finalize sample: the 4 planes of a 2-ring sub-scanner with the full
    # view x radial x TOF extent
    sub = np.random.default_rng(0).integers(0, 1 << 36, size=(4, sc.n_views, sc.n_rad, sc.n_tof))
    t = time.perf_counter()
    oracle.finalize(sub, 2, sens=sens[:4], sigma=(2.0, 2.0, 2.0), scale=1.0 / n)
    per_bin = (time.perf_counter() - t) / sub.size
    step_s = per_h * n + per_bin * sc.n_bins
    return {"value": n / step_s, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{m} histories of the workload on {cores} threads ({per_h * 1e6:.3f} us each) + "
                      f"finalize of {sub.size} bins ({per_bin * 1e9:.1f} ns each), extrapolated to "
                      f"{n} histories and {sc.n_bins} bins per step"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import oracle
    sc, mats, ph, lut, sens, workload = workload_inputs(a)
    n = int(a.histories)
    for i in range(a.warmup):  # untimed: a short oracle run per warm-up step
        oracle.simulate(sc, mats, ph, lut, 100 + i, 0, 2000, threads=os.cpu_count() or 1)
    vals, walls = [], []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        vals.append(cpu_baseline(sc, mats, ph, lut, sens, n, budget_s=8.0)["value"])
        walls.append(time.perf_counter() - t0)
    v = float(np.median(vals))
    # each step is a bounded sample of the workload (histories and a finalize
    # share, both linear in the step's size), so ms_per_step is the sample's
    # measured wall time and value the sample's rate: histories/s of the workload
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * float(np.mean(walls)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": step_config(sc, workload, n, 1),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "each step: a bounded oracle sample (about 8 s: histories of the workload and "
                                       "a finalize of a 4-plane slab), timed per history and per bin, the rate "
                                       "extrapolated to the step's 1e9 histories and its full sinogram"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------------------
# precision study: FP32 / FP16 / BF16 LUT at low count levels against a
# high-count FP32 reference, after smoothing (relative RMS over all bins)
# ---------------------------------------------------------------------------
def run_precision(a):
    import torch
    import paper_2509_05047_gb300 as psc
    from paper_2509_05047_gb300 import build as B
    B.build()
    if a.precision_workload == "paper":
        sc, mats, ph, lut, sens = build_inputs(a.rings, a.tof_bins)
        workload = WORKLOAD
    else:
        sc, mats, ph = W.scanner_tiny(), W.standard_materials(), W.phantom_water_cylinder()
        lut, sens = W.lut_tiny(sc), W.sensitivity_uniform(sc.lor_shape, seed=1)
        workload = WORKLOAD_SMALL
    dev = torch.device("cuda", 0)
    ctx = psc.psc_create(0)
    s_id = psc.psc_load_scanner(ctx, psc.scanner_desc(sc))
    m_id = psc.psc_load_materials(ctx, psc.materials_desc(mats).desc)
    p_id = psc.psc_load_phantom(ctx, psc.phantom_desc(ph).desc, m_id)
    luts = {name: psc.psc_load_lut(ctx, psc.lut_desc(lut, dt).desc)
            for name, dt in (("f32", psc.PSC_LUT_F32), ("f16", psc.PSC_LUT_F16), ("bf16", psc.PSC_LUT_BF16))}
    sn_id = psc.psc_load_sinogram(ctx, s_id, sens, per_lor=True)
    a_id = psc.psc_acc_create(ctx, s_id)
    sh = torch.cuda.current_stream(dev).cuda_stream
    sigma = tuple(a.sigma)

    def estimate(n, lut_id, seed, out):
        psc.psc_acc_zero(ctx, a_id, sh)
        done = 0
        while done < n:                       # 1e9-history launches
            k = min(int(1e9), n - done)
            psc.psc_simulate(ctx, psc.sim_args(seed, done, k, s_id, p_id, a_id, lut=lut_id), stream=sh)
            done += k
        psc.psc_finalize(ctx, psc.finalize_args(a_id, sens=sn_id, sigma=sigma, scale=1.0 / n), out, sh)
        torch.cuda.synchronize()

    def rel_rms(x, ref):
        num, den = 0.0, 0.0
        xf, rf = x.view(-1), ref.view(-1)
        for i in range(0, xf.numel(), 1 << 28):
            d = xf[i:i + (1 << 28)] - rf[i:i + (1 << 28)]
            num += float((d * d).sum())
            den += float((rf[i:i + (1 << 28)] ** 2).sum())
        return math.sqrt(num / den) if den > 0 else float("nan")

    n_ref = int(a.reference_histories)
    ref = torch.empty(sc.shape, dtype=torch.float64, device=dev)
    t = time.perf_counter()
    estimate(n_ref, luts["f32"], 777, ref)
    t_ref = time.perf_counter() - t
    out = torch.empty(sc.shape, dtype=torch.float64, device=dev)
    base = torch.empty(sc.shape, dtype=torch.float64, device=dev)
    rows = []
    for n in (int(1e7), int(1e8)):
        estimate(n, luts["f32"], 4242, base)
        for name in ("f32", "f16", "bf16"):
            estimate(n, luts[name], 4242, out)
            rows.append({"histories": n, "lut": name, "rel_rms_vs_reference": rel_rms(out, ref),
                         "rel_rms_vs_f32_same_histories": rel_rms(out, base)})
    psc.psc_destroy(ctx)
    return {"mode": "precision", "workload": workload, "reference_histories": n_ref,
            "reference_seconds": t_ref, "smoothing_sigma_bins": sigma,
            "metric": "relative RMS sqrt(sum (A-B)^2 / sum B^2) over all bins after smoothing",
            "rows": rows}


# ---------------------------------------------------------------------------
# accuracy against history budget (the 1 % relative-RMS clause)
# ---------------------------------------------------------------------------
def run_accuracy(a):
    """Relative RMS after smoothing (the paper's kernel widths by default)
    against a reference whose own noise is measured: the reference is the
    mean of two independent halves (seeds), so RMS(half1, half2) / 2 is its
    own relative RMS noise, and an estimate's error is sqrt(RMS(A, ref)^2 -
    noise_ref^2).  Budgets grow until the corrected error is below 1 %."""
    import torch
    import paper_2509_05047_gb300 as psc
    from paper_2509_05047_gb300 import build as B
    B.build()
    sc, mats, ph = W.scanner_tiny(), W.standard_materials(), W.phantom_water_cylinder()
    lut, sens = W.lut_tiny(sc), W.sensitivity_uniform(sc.lor_shape, seed=1)
    dev = torch.device("cuda", 0)
    ctx = psc.psc_create(0)
    s_id = psc.psc_load_scanner(ctx, psc.scanner_desc(sc))
    m_id = psc.psc_load_materials(ctx, psc.materials_desc(mats).desc)
    p_id = psc.psc_load_phantom(ctx, psc.phantom_desc(ph).desc, m_id)
    l_id = psc.psc_load_lut(ctx, psc.lut_desc(lut).desc)
    sn_id = psc.psc_load_sinogram(ctx, s_id, sens, per_lor=True)
    a_id = psc.psc_acc_create(ctx, s_id)
    sh = torch.cuda.current_stream(dev).cuda_stream
    sigma = tuple(a.sigma)
    B_LAUNCH = int(2e9)

    def estimate(n, seed, out):
        psc.psc_acc_zero(ctx, a_id, sh)
        done = 0
        while done < n:
            k = min(B_LAUNCH, n - done)
            psc.psc_simulate(ctx, psc.sim_args(seed, done, k, s_id, p_id, a_id, lut=l_id), stream=sh)
            done += k
        psc.psc_finalize(ctx, psc.finalize_args(a_id, sens=sn_id, sigma=sigma, scale=1.0 / n), out, sh)
        torch.cuda.synchronize()

    def rms2(x, ref):
        d = (x - ref).view(-1)
        return float((d * d).sum()) / float((ref.view(-1) ** 2).sum())

    n_half = int(a.reference_histories) // 2
    h1 = torch.empty(sc.shape, dtype=torch.float64, device=dev)
    h2 = torch.empty_like(h1)
    t = time.perf_counter()
    estimate(n_half, 9001, h1)
    estimate(n_half, 9002, h2)
    t_ref = time.perf_counter() - t
    ref = (h1 + h2) * 0.5
    noise_ref2 = rms2(h1, h2) / 4.0          # RMS(h1 - h2)^2 = 2 noise(half)^2 = 4 noise(ref)^2
    del h1, h2
    out = torch.empty_like(ref)
    rows = []
    for n in (int(1e8), int(1e9), int(1e10), int(3e10), int(1e11)):
        t = time.perf_counter()
        estimate(n, 4242, out)
        dt = time.perf_counter() - t
        r2 = rms2(out, ref)
        rows.append({"histories": n, "rel_rms_vs_reference": math.sqrt(r2),
                     "rel_rms_corrected": math.sqrt(max(r2 - noise_ref2, 0.0)), "seconds": round(dt, 3)})
    psc.psc_destroy(ctx)
    # the error falls as 1/sqrt(n): the budget for 1 % from the largest budget
    last = rows[-1]
    need = last["histories"] * (last["rel_rms_corrected"] / 0.01) ** 2
    return {"mode": "accuracy", "workload": WORKLOAD_SMALL, "smoothing_sigma_bins": sigma,
            "reference_histories": 2 * n_half, "reference_seconds": round(t_ref, 2),
            "reference_rel_rms_noise": math.sqrt(noise_ref2),
            "metric": "relative RMS sqrt(sum (A-B)^2 / sum B^2) over all bins after smoothing; corrected: "
                      "sqrt(RMS^2 - reference noise^2), the reference noise from its two independent halves",
            "rows": rows, "histories_for_1pct": need}


# ---------------------------------------------------------------------------
# batched / served requests against plain sequential requests
# ---------------------------------------------------------------------------
def _request_mix(a, served):
    """(kind, phantom builder key, budget, seed) per request.  batched: one
    request per seeded ellipsoid torso (96^3-class to 192x192x120) on the
    small scanner (288 x 16 crystals); served: 5-iteration chains mixing the
    small configuration, the paper-scale torso and scanner, and the
    batched-style torsos."""
    rng = np.random.default_rng(2025)
    lo, hi = 6.0, 9.0
    out = []
    if not served:
        dims = W.batched_phantom_dims(a.requests)
        for i, d in enumerate(dims):
            n = int(a.budget_scale * 10 ** rng.uniform(lo, hi))
            out.append({"kind": "torso", "dims": d, "seed": 100 + i, "n": max(n, 1000), "chain": i, "it": 0})
        return out
    for c in range(a.requests):
        kind = ["tiny", "paper", "torso"][c % 3]
        n = max(int(a.budget_scale * 10 ** rng.uniform(lo, hi)), 1000)
        d = W.batched_phantom_dims(1, seed=500 + c)[0]
        for it in range(5):
            out.append({"kind": kind, "dims": d, "seed": 1000 * c + it, "n": n, "chain": c, "it": it})
    return out


def run_requests(a, served=None, chains=None, max_active=None):
    """Plain sequential requests against the request server on one request
    mix.  batched (served False): every request arrives at t = 0.  served:
    chains of 5 iterations, each chain starting at a Poisson arrival and
    issuing its next iteration when the previous estimate is back.  Both arms
    see the same arrivals: the plain arm is one worker that takes requests in
    arrival order and runs each alone with cold residency (phantom load with
    its alias table, accumulator allocation, simulate, finalize, free), so its
    latency includes the wait behind earlier requests; the served arm keeps
    phantoms resident and batches the active requests in each launch."""
    import queue
    import threading
    import torch
    import paper_2509_05047_gb300 as psc
    from paper_2509_05047_gb300 import build as B
    B.build()
    served = (a.mode == "served") if served is None else served
    n_chains = a.requests if chains is None else chains
    max_active = a.max_active if max_active is None else max_active
    a2 = argparse.Namespace(**vars(a))
    a2.requests = n_chains
    dev = torch.device("cuda", 0)
    mats = W.standard_materials()
    sc_tiny, sc_paper = W.scanner_tiny(), W.scanner_signa()
    mix = _request_mix(a2, served)
    phantoms = {}
    for r in mix:
        key = (r["kind"], r["dims"], r["chain"])
        if key not in phantoms:
            if r["kind"] == "tiny":
                phantoms[key] = W.phantom_water_cylinder()
            elif r["kind"] == "paper":
                phantoms[key] = W.phantom_torso()
            else:
                phantoms[key] = W.phantom_random_torso(7 + r["chain"], r["dims"],
                                                        W.batched_phantom_voxel(r["dims"]))
    rng = np.random.default_rng(3)
    for r in mix:     # each chain iteration brings a new activity image
        ph = phantoms[(r["kind"], r["dims"], r["chain"])]
        r["activity"] = (ph.activity * rng.uniform(0.7, 1.3, ph.activity.shape)).astype(np.float32)
    sigma = (2.0, 2.0, 2.0)

    # accumulators and resident objects share a 140 GB budget (three paper-scale
    # accumulators), the rest of HBM holds outputs and the smoothing buffer
    ctx = psc.psc_create(0, int(140e9))
    s_tiny = psc.psc_load_scanner(ctx, psc.scanner_desc(sc_tiny))
    s_paper = psc.psc_load_scanner(ctx, psc.scanner_desc(sc_paper))
    m_id = psc.psc_load_materials(ctx, psc.materials_desc(mats).desc)
    l_tiny = psc.psc_load_lut(ctx, psc.lut_desc(W.lut_tiny(sc_tiny)).desc)
    l_paper = psc.psc_load_lut(ctx, psc.lut_desc(W.lut_signa(sc_paper)).desc)
    sn_tiny = psc.psc_load_sinogram(ctx, s_tiny, W.sensitivity_uniform(sc_tiny.lor_shape, seed=1), True)
    sn_paper = psc.psc_load_sinogram(ctx, s_paper, W.sensitivity_uniform(sc_paper.lor_shape, seed=1), True)
    scan = {"tiny": (s_tiny, l_tiny, sn_tiny, sc_tiny), "torso": (s_tiny, l_tiny, sn_tiny, sc_tiny),
            "paper": (s_paper, l_paper, sn_paper, sc_paper)}
    okind = lambda kind: "paper" if kind == "paper" else "tiny"   # output shape of a request
    stream = torch.cuda.current_stream(dev).cuda_stream
    total_h = sum(r["n"] for r in mix)
    arrivals = np.cumsum(np.random.default_rng(4).exponential(1.0 / a.rate, size=len(mix))) if served \
        else np.zeros(len(mix))
    by_chain = {}
    for i, r in enumerate(mix):
        by_chain.setdefault(r["chain"], []).append(i)
    starts = arrivals[[by_chain[c][0] for c in sorted(by_chain)]] if served else np.zeros(len(by_chain))
    pct = lambda v, q: float(np.percentile(np.asarray(v), q))

    def drive(submit_and_wait):
        """Chain workers: each chain starts at its arrival and issues its next
        iteration when the previous one is back.  Returns (seconds, latencies)."""
        lat = []
        lk = threading.Lock()
        t0 = time.perf_counter()

        def worker(c, first_arrival):
            wait = first_arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            for i in by_chain[c]:
                ts = time.perf_counter()
                submit_and_wait(mix[i])
                with lk:
                    lat.append(time.perf_counter() - ts)

        ths = [threading.Thread(target=worker, args=(c, float(st))) for c, st in zip(sorted(by_chain), starts)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        return time.perf_counter() - t0, lat

    # ---- plain: one worker, requests in arrival order, each alone and cold ----
    outs = {"tiny": torch.empty(sc_tiny.shape, dtype=torch.float64, device=dev),
            "paper": torch.empty(sc_paper.shape, dtype=torch.float64, device=dev)}
    service = []

    def plain_one(r):
        ts = time.perf_counter()
        s_id, l_id, sn_id, sc = scan[r["kind"]]
        ph = phantoms[(r["kind"], r["dims"], r["chain"])]
        desc = psc.phantom_desc(W.Phantom(ph.dims, ph.voxel, ph.origin, ph.material, ph.density, r["activity"]))
        p_id = psc.psc_load_phantom(ctx, desc.desc, m_id)
        acc = psc.psc_acc_create(ctx, s_id)
        psc.psc_simulate(ctx, psc.sim_args(r["seed"], 0, r["n"], s_id, p_id, acc, lut=l_id), stream=stream)
        psc.psc_finalize(ctx, psc.finalize_args(acc, sens=sn_id, sigma=sigma, scale=1.0 / r["n"]),
                         outs[okind(r["kind"])], stream)
        torch.cuda.synchronize()
        psc.psc_unload(ctx, acc)
        psc.psc_unload(ctx, p_id)
        service.append(time.perf_counter() - ts)

    torch.cuda.synchronize()
    if served:
        q = queue.Queue()

        def plain_server():
            while True:
                item = q.get()
                if item is None:
                    return
                plain_one(item[0])
                item[1].set()

        srv = threading.Thread(target=plain_server)
        srv.start()

        def plain_submit(r):
            done = threading.Event()
            q.put((r, done))
            done.wait()

        t_plain, plain_lat = drive(plain_submit)
        q.put(None)
        srv.join()
    else:   # every request arrives at t = 0: the worker takes them in the mix's order
        t0 = time.perf_counter()
        plain_lat = []
        for r in mix:
            plain_one(r)
            plain_lat.append(time.perf_counter() - t0)
        t_plain = time.perf_counter() - t0

    # ---- served: resident phantoms, request server ----
    del outs
    torch.cuda.empty_cache()
    pids = {key: psc.psc_load_phantom(ctx, psc.phantom_desc(ph).desc, m_id) for key, ph in phantoms.items()}
    n_out = max_active + 2
    pool = {"tiny": [torch.empty(sc_tiny.shape, dtype=torch.float64, device=dev) for _ in range(n_out)],
            "paper": [torch.empty(sc_paper.shape, dtype=torch.float64, device=dev) for _ in range(2)]}
    free_out = {k: list(range(len(v))) for k, v in pool.items()}
    torch.cuda.synchronize()
    cond = threading.Condition(threading.Lock())

    def take_out(kind):
        k = okind(kind)
        with cond:
            while not free_out[k]:
                cond.wait()
            return k, free_out[k].pop()

    def give_out(k, j):
        with cond:
            free_out[k].append(j)
            cond.notify_all()

    def served_submit(r):
        s_id, l_id, sn_id, sc = scan[r["kind"]]
        k, j = take_out(r["kind"])
        t = psc.psc_submit(ctx, psc.request(s_id, pids[(r["kind"], r["dims"], r["chain"])], pool[k][j],
                                            r["n"], r["seed"], lut=l_id, sens=sn_id, sigma=sigma,
                                            scale=1.0 / r["n"], activity=r["activity"]))
        psc.psc_wait(ctx, t)
        give_out(k, j)

    psc.psc_server_start(ctx, max_active=max_active, epoch_histories=int(2e8), min_slice=65536)
    t_served, lat = drive(served_submit)
    psc.psc_server_stop(ctx)

    # ---- batched: every request in one persistent launch with an autotuned
    # schedule (resident phantoms; each request's new activity image gets its
    # alias table on one of 16 threads, inside the timed region) ----
    one = None
    if not served:
        from concurrent.futures import ThreadPoolExecutor
        keys = [(r["kind"], r["dims"], r["chain"]) for r in mix]
        accs = [psc.psc_acc_create(ctx, scan[r["kind"]][0]) for r in mix]
        out1 = pool["tiny"][0]

        def one_launch():
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with ThreadPoolExecutor(16) as ex:
                list(ex.map(lambda i: psc.psc_update_activity(ctx, pids[keys[i]], mix[i]["activity"]),
                            range(len(mix))))
            for acc in accs:
                psc.psc_acc_zero(ctx, acc, stream)
            sched = psc.psc_simulate_batch_tuned(
                ctx, [psc.sim_args(r["seed"], 0, r["n"], scan[r["kind"]][0], pids[k], acc, lut=scan[r["kind"]][1])
                      for r, k, acc in zip(mix, keys, accs)], stream=stream)
            for r, acc in zip(mix, accs):
                psc.psc_finalize(ctx, psc.finalize_args(acc, sens=scan[r["kind"]][2], sigma=sigma,
                                                        scale=1.0 / r["n"]), out1, stream)
            torch.cuda.synchronize()
            return time.perf_counter() - t0, sched

        t_first, s_first = one_launch()
        t_again, s_again = one_launch()

        # the same GPU step (zero, the tuned launch on the cached schedule, finalizes)
        # captured once into a CUDA graph and replayed; the activity updates stay on
        # the host, before each replay
        batch_args = [psc.sim_args(r["seed"], 0, r["n"], scan[r["kind"]][0], pids[k], acc, lut=scan[r["kind"]][1])
                      for r, k, acc in zip(mix, keys, accs)]

        def gpu_step():
            sh2 = torch.cuda.current_stream().cuda_stream
            for acc in accs:
                psc.psc_acc_zero(ctx, acc, sh2)
            psc.psc_simulate_batch_tuned(ctx, batch_args, stream=sh2)
            for r, acc in zip(mix, accs):
                psc.psc_finalize(ctx, psc.finalize_args(acc, sens=scan[r["kind"]][2], sigma=sigma,
                                                        scale=1.0 / r["n"]), out1, sh2)

        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side, capture_error_mode="thread_local"):
            gpu_step()
        torch.cuda.synchronize()

        def graph_step():
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with ThreadPoolExecutor(16) as ex:
                list(ex.map(lambda i: psc.psc_update_activity(ctx, pids[keys[i]], mix[i]["activity"]),
                            range(len(mix))))
            graph.replay()
            torch.cuda.synchronize()
            return time.perf_counter() - t0

        t_graph = min(graph_step() for _ in range(2))
        del graph
        one = {"seconds": round(t_first, 4), "histories_per_s": total_h / t_first,
               "speedup_vs_plain": t_plain / t_first,
               "seconds_cached_schedule": round(t_again, 4), "histories_per_s_cached": total_h / t_again,
               "speedup_vs_plain_cached": t_plain / t_again,
               "seconds_graph": round(t_graph, 4), "histories_per_s_graph": total_h / t_graph,
               "speedup_vs_plain_graph": t_plain / t_graph,
               "schedule": {k: (round(v, 1) if isinstance(v, float) else v) for k, v in s_first.items()},
               "note": "first call: the autotuner's probes run the first 6/48 of every budget with candidate "
                       "schedules, the choice runs the rest; second call: the cached choice; graph: the GPU "
                       "part captured once into a CUDA graph and replayed after the host's alias builds"}
    psc.psc_destroy(ctx)
    return {"mode": "served" if served else "batched", "requests": len(mix), "histories": total_h,
            "budget_scale": a.budget_scale,
            "plain": {"seconds": round(t_plain, 4), "histories_per_s": total_h / t_plain,
                      "p50_latency_s": round(pct(plain_lat, 50), 4), "p99_latency_s": round(pct(plain_lat, 99), 4),
                      "p50_service_s": round(pct(service, 50), 4)},
            "served": {"seconds": round(t_served, 4), "histories_per_s": total_h / t_served,
                       "p50_latency_s": round(pct(lat, 50), 4), "p99_latency_s": round(pct(lat, 99), 4),
                       "max_active": max_active, "arrival_rate_per_s": a.rate if served else None},
            "speedup": t_plain / t_served,
            "one_launch": one,
            "latency": "from submission to the estimate in device memory; plain requests wait for the ones "
                       "before them",
            "note": "served results are bit-identical to the same requests alone (tests/test_gpu_server.py)"}


# ---------------------------------------------------------------------------
# post-processing calls on the paper-scale sinogram
# ---------------------------------------------------------------------------
def run_postproc(a):
    import torch
    import paper_2509_05047_gb300 as psc
    from paper_2509_05047_gb300 import build as B
    B.build()
    sc = W.scanner_signa()
    if a.rings:   # profiling case: fewer rings, the same planes' layout
        sc = W.Scanner(sc.radius, sc.n_crystals, a.rings, sc.ring_pitch, sc.module_t, sc.module_a,
                       sc.e_lo, sc.e_hi, sc.n_tof, sc.tof_bin_mm, sc.tof_sigma_mm)
    ctx = psc.psc_create(0)
    s_id = psc.psc_load_scanner(ctx, psc.scanner_desc(sc))
    a_id, o_id = psc.psc_acc_create(ctx, s_id), psc.psc_acc_create(ctx, s_id)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    # a dense synthetic accumulator (every bin non-zero, as after a long run)
    acc = torch.empty(sc.n_bins, dtype=torch.int64, device="cuda")
    acc.random_(1 << 20, 1 << 36, generator=torch.Generator(device="cuda").manual_seed(1))
    psc.psc_acc_write(ctx, a_id, acc, sh)
    del acc
    out = torch.empty(sc.shape, dtype=torch.float64, device="cuda")
    mashed = torch.empty((sc.n_planes, sc.n_views // 2, sc.n_rad, sc.n_tof), dtype=torch.int64, device="cuda")
    ops = {
        "rotate_sum_step16": (lambda: psc.psc_acc_rotate_sum(ctx, a_id, 16, o_id, sh), 16),
        "mash_views2": (lambda: psc.psc_acc_mash(ctx, a_id, 2, 1, mashed, sh), 12),
        "norm_sinogram_sigma4": (lambda: psc.psc_norm_sinogram(ctx, a_id, (4.0, 4.0, 4.0), out, sh), 32),
    }
    peaks, src = measured_peaks()
    span_out = torch.empty((psc.psc_acc_span(ctx, a_id, 3),) + sc.shape[1:], dtype=torch.int64, device="cuda")
    ops["span3"] = (lambda: psc.psc_acc_span(ctx, a_id, 3, span_out, sh), 8 + 8 * span_out.shape[0] / sc.n_planes)
    res = {"mode": "postproc", "workload": f"paper-scale sinogram {sc.n_planes}x{sc.n_views}x{sc.n_rad}x{sc.n_tof} "
                                           f"({sc.n_bins / 1e9:.2f}e9 bins), dense int64",
           "hbm_peak_gbs": peaks["hbm_gbs"], "ops": {}}
    for name, (f, bytes_per_bin) in ops.items():
        for _ in range(2):
            f()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            f()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        gbs = bytes_per_bin * sc.n_bins / (ms / 1e3) / 1e9
        res["ops"][name] = {"ms": round(ms, 3), "algorithmic_bytes_per_bin": bytes_per_bin,
                            "achieved_gbs": round(gbs, 1), "frac_of_hbm": round(gbs / peaks["hbm_gbs"], 3)}
    psc.psc_destroy(ctx)
    return res


def main():
    a = parse()
    if a.mode == "postproc":
        print(json.dumps(run_postproc(a)))
        return
    if a.mode in ("batched", "served"):
        print(json.dumps(run_requests(a)))
        return
    if a.mode == "precision":
        print(json.dumps(run_precision(a)))
        return
    if a.mode == "accuracy":
        print(json.dumps(run_accuracy(a)))
        return
    res = run_reference(a) if a.impl == "reference" else run_native(a)
    if res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
