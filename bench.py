"""Benchmark of the GB300 quasi-3D dual-solver PIC step.

Workload (default): the 4000 x 400 LWFA/DLA box, modes m = 0, 1, dz = 0.2,
dr = 0.8, 32 particles per cell (51.2M macroparticles), moving window at c,
dual solver with 16 coefficients, dt = 0.9 x its stability limit, FP32 push
and solve with int64 fixed-point current.  One step = Faraday, gather + push +
deposit, J decode + J_z filter, Ampere, window shift/injection and the particle
sort.  Synthetic inputs (seeded plasma lattice + Gaussian laser); the box's
1.8 GB of particles exceed the 129 MB L2, so no flush is needed between steps.

Prints one JSON line: value = particle-steps/s of the whole step (all ranks),
with cell-updates/s, the roofline of the gather+push+deposit kernel, the
FP64 oracle timed on the host cores (cpu_baseline), an end-to-end number
through the C ABI with host buffers, SM clocks sampled during the timed
region, and the number of kernels launched.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference]
Multi-GPU (torchrun): every rank runs an independent replica of the box
("replicas only"; weak scaling), timed between barriers, max over ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "particle-steps/s (gather+push+deposit) + solver cell-updates/s, FP32 vs FP64"
# algorithmic bytes of gather+push+deposit per particle-step at P particles per
# cell: particle read 36 B + write 32 B, plus per cell E and Bbar (72 B read)
# and the int64 current (72 B read-modify-write = 144 B), amortised over P
GPD_BYTES_PER_PARTICLE = 68.0
GPD_BYTES_PER_CELL = 72.0 + 144.0


def kernel_bytes(name, w, particles, launches, nkeys, tile=(16, 8)):
    """Algorithmic bytes one kernel class moves over `launches` launches (FP32
    path, np = 2M+1 mode parts, cells = nz nr):
    - faraday: read E, B; write B, Bbar: 4 x 12 np B per cell;
    - ampere: read E, B, J; write E: 4 x 12 np B per cell;
    - jz_filter: read and write J_z: 2 x 4 np B per cell;
    - j_decode: read the int64 tile blocks that cover a cell (3 np words per node,
      (TZ+5)(TR+5) nodes per TZ x TR tile) and write the FP32 current (12 np B);
    - gather_push_deposit: 68 B per particle + 216 B per cell (as above);
    - sort: per sort, 76 B per particle (cell read twice, record read and
      written, cell written) and 24 B per key (counts and offsets passes)."""
    np_ = 2 * w["n_modes"] - 1
    cells = w["nz"] * w["nr"]
    tz, tr = tile
    per = {
        "faraday": 48.0 * np_ * cells,
        "ampere": 48.0 * np_ * cells,
        "jz_filter": 8.0 * np_ * cells,
        "j_decode": (24.0 * np_ * (tz + 5) * (tr + 5) / (tz * tr) + 12.0 * np_) * cells,
        "gather_push_deposit": GPD_BYTES_PER_PARTICLE * particles + GPD_BYTES_PER_CELL * cells,
        "sort": 76.0 * particles + 24.0 * nkeys,
    }
    return per[name] * launches if name in per else None


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = "/tmp/qpic_clocks_%d.csv" % os.getpid()

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _measured_traffic(workload, kernel_rev):
    """DRAM bytes per k_gpd launch from the committed ncu summary, when it was
    taken on this workload with this kernel revision; else None."""
    path = os.path.join(ROOT, "profiles", "gpd_%s_dram_traffic.md" % workload)
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("|"):
            k, _, v = line.partition(":")
            kv[k.strip()] = v.strip()
    if kv.get("kernel_rev") != kernel_rev or kv.get("workload") != workload:
        return None
    try:
        return int(kv["bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _make_sim(q, w, stream, track_work=False, precision=None):
    kw = {} if precision is None else {"precision": precision}
    return q.Sim(w["nz"], w["nr"], w["dz"], w["dr"], n_modes=w["n_modes"], solver=w["solver"],
                 periodic=w["periodic"], moving_window=w["moving_window"], stream=stream,
                 track_work=track_work, seed=w["plasma"]["seed"], **kw)


def _init_state(sim, w):
    pl, la = w["plasma"], w["laser"]
    sim.load_plasma(pl["n0"], pl["z_start"], pl["ramp_len"], pl["ppc"])
    sim.add_laser(la["a0"], la["w0"], la["fwhm"], la["z_centroid"], la["z_focus"])


def reduced_leg(q, torch, stream, args):
    """The reduced model of Eq. 8 (FP64 Dormand-Prince, one thread per electron) on
    a synthetic bunch; the oracle timed on a small sample unless --no-cpu."""
    nr_e, st_e = args.reduced_electrons, args.reduced_steps
    # Appendix A's bunch and parameters, in units of the local laser frequency
    # (omega0 = v_phi k_z = 12.17 omega_p); k_perp = 2.4/(R + c/omega_p) with R
    # standing for the mean bubble radius at the bunch
    P = synth.REDUCED_PAPER
    wp = 1.0 / (P["v_phi"] * P["kz_over_wp"])
    y0 = list(synth.reduced_bunch(8, nr_e, v_g=P["v_g"], wp=wp, R_over_lp=P["R_over_lp"]))
    par = (P["a0"], wp, 2.4 * wp / (P["R_over_lp"] + 1.0), P["v_phi"])   # a0, omega_p, k_perp, v_phi
    dev = [torch.tensor(v, dtype=torch.float64, device="cuda") for v in y0]
    ptrs = [d.data_ptr() for d in dev]
    sh = stream.cuda_stream
    q.reduced_integrate_device(ptrs, nr_e, *par, 0.0, 0.05, 5, stream=sh)     # warm-up
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    q.reduced_integrate_device(ptrs, nr_e, *par, 0.25, 0.05, st_e, stream=sh)
    g1.record(stream)
    torch.cuda.synchronize()
    msr = g0.elapsed_time(g1)
    ocpu = None
    if not args.no_cpu:
        from oracle import reduced as R             # the oracle, for this leg's CPU baseline only
        ns = 1000
        t0c = time.perf_counter()
        R.integrate(*[v[:ns] for v in y0], *par, 0.0, 0.05, 50)
        tc = time.perf_counter() - t0c
        ocpu = {"value": ns * 50 / tc, "unit": "electron-steps/s", "cores": 1, "kind": "oracle",
                "sample": "1000 electrons x 50 steps, numpy FP64"}
    out = {"value": nr_e * st_e / (msr / 1e3), "unit": "electron-steps/s", "electrons": nr_e,
           "steps": st_e, "ms": msr, "dtype": "f64", "cpu_baseline": ocpu,
           "note": "Eq. 8 with Appendix A's bunch and parameters (a0 2.8, v_phi 1.002565, "
                   "k_z 12.14 omega_p, R 3 c/omega_p), fifth-order Dormand-Prince at dt 0.05 / omega0"}
    if args.reduced_divergence_electrons > 0:
        out["staggering"] = reduced_divergence(q, torch, stream, args.reduced_divergence_electrons, par, wp)
    return out


def reduced_divergence(q, torch, stream, n, par, wp):
    """Sec. IV.A: the time-staggering factor cos(omega0 dt/2) on the laser's
    magnetic terms (dt the paper's 3D Yee step, 0.01875 / omega_p) widens the
    divergence angle theta_x = atan(u_x / u_z) of the most energetic
    electrons.  The Appendix A bunch, injected uniformly over 200 / omega_p,
    is integrated over the paper's 430 um plateau (3315 c / omega0 at
    815 nm) with and without the factor."""
    P = synth.REDUCED_PAPER
    dt = 0.05
    y0 = synth.reduced_bunch(9, n, v_g=P["v_g"], wp=wp, R_over_lp=P["R_over_lp"])
    steps = int(round(3315.0 / dt))
    start = np.random.default_rng([9, 1]).integers(0, int(round(200.0 / wp / dt)), n).astype(np.int32)
    bfac = float(np.cos(0.5 * 0.01875 / wp))
    res = {}
    ds = torch.tensor(start, dtype=torch.int32, device="cuda")
    for name, b in (("without", 1.0), ("with", bfac)):
        dev = [torch.tensor(v, dtype=torch.float64, device="cuda") for v in y0]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        q.reduced_integrate_device([d.data_ptr() for d in dev], n, *par, 0.0, dt, steps,
                                   stream=stream.cuda_stream, bfac=b, start_ptr=ds.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        x, zeta, ux, uz = (d.cpu().numpy() for d in dev)
        gamma = np.sqrt(1 + ux ** 2 + uz ** 2)
        top = gamma >= np.quantile(gamma, 0.9)                # the most energetic 10%
        th = np.arctan2(ux, uz)
        res[name] = {"bfac": b, "ms": e0.elapsed_time(e1), "gamma_top10_mean": float(gamma[top].mean()),
                     "theta_rms_top10_mrad": float(1e3 * np.sqrt(np.mean(th[top] ** 2))),
                     "theta_rms_all_mrad": float(1e3 * np.sqrt(np.mean(th ** 2)))}
    res["theta_rms_top10_ratio"] = res["with"]["theta_rms_top10_mrad"] / res["without"]["theta_rms_top10_mrad"]
    res["electrons"], res["steps"] = n, steps
    return res


def batch_scan(q, torch, stream, nruns, steps, seed=5):
    """Parameter scan of independent periodic runs (grids 256-1024 x 32-128,
    n 0.003-0.02, a0 1-4, ppc 8/16/32; run k draws from a generator seeded
    (seed, k)).  The tile shape, sort period (2 or 4) and particles per
    thread (4 or 8) of each particles-per-cell class come from the autotuner
    (a batch of four 512 x 64 runs of that class).  The same runs are stepped one
    after another, then together as one graph-launched batch whose particle
    phase is one persistent launch per group of runs.  Returns aggregate
    particle-steps/s of both."""
    from paper_2303_12874_gb300 import autotune
    tiles = {}
    for ppc_ in ((2, 2, 2), (2, 2, 4), (2, 2, 8)):
        def make(tz, tr, sp, ppt):
            return q.Sim(512, 64, 0.2, 0.5, stream=stream, tile_z=tz, tile_r=tr, sort_period=sp,
                         particles_per_thread=ppt)

        def init(sim, ppc_=ppc_):
            sim.load_plasma(0.01, 0.0, 0.0, ppc_)
            sim.add_laser(2.0, 8.0, 15.0, 51.2, 51.2)
        tz, tr, sp, ppt, _ = autotune.tune(make, init, 512, 64, 2, int(np.prod(ppc_)), steps=8, warmup=4,
                                           sort_periods=(2, 4), batch_copies=4,
                                           particles_per_thread=(8, 16))
        tiles[ppc_] = (tz, tr, sp, ppt)
    sims, npart = [], []
    for k in range(nruns):
        rng = np.random.default_rng([seed, k])
        nz = int(rng.integers(256, 1025)) // 16 * 16
        nr = int(rng.integers(32, 129))
        n0 = float(rng.uniform(0.003, 0.02))
        a0 = float(rng.uniform(1.0, 4.0))
        ppc = [(2, 2, 2), (2, 2, 4), (2, 2, 8)][int(rng.integers(0, 3))]
        sim = q.Sim(nz, nr, 0.2, 0.5, stream=stream, seed=seed * 1000 + k, tile_z=tiles[ppc][0],
                    tile_r=tiles[ppc][1], sort_period=tiles[ppc][2], particles_per_thread=tiles[ppc][3])
        sim.load_plasma(n0, 0.0, 0.0, ppc)
        zc = 0.5 * nz * 0.2
        sim.add_laser(a0, 8.0, 15.0, zc, zc)
        sims.append(sim)
        npart.append(sim.diag()["particles"])
    total = float(sum(npart))
    for sm in sims:
        sm.step(2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for sm in sims:
        sm.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    batch = q.Batch(sims, stream=stream)
    cycle = batch.cycle
    batch.step(batch.cycle)
    torch.cuda.synchronize()
    e0.record(stream)
    nb = max(cycle, steps - steps % cycle)
    batch.step(nb)
    e1.record(stream)
    torch.cuda.synchronize()
    bat_ms = e0.elapsed_time(e1)
    batch.close()
    for sm in sims:
        sm.close()
    return {"runs": nruns, "particles": int(total), "steps": steps,
            "tiles": {"ppc %d" % int(np.prod(k)): "%dx%d sort %d, %d particles per thread" % v
                      for k, v in tiles.items()},
            "cycle": cycle,
            "sequential": total * steps / (seq_ms / 1e3), "batched_graph": total * nb / (bat_ms / 1e3),
            "speedup": (nb / bat_ms) / (steps / seq_ms), "unit": "particle-steps/s"}


def oracle_sample(w, dt, nz_sample, steps, threads=1):
    """The FP64 oracle, as it stands, on a z-slab of the workload: the same
    nr, dz, dr, dt, plasma and ppc over nz_sample columns (periodic).  With
    threads > 1 its multi-threaded mode (4 particle ranges per thread).
    Returns (particle-steps/s, particles, seconds)."""
    import oracle
    from oracle import coeffs as C
    from oracle import setup as S
    pl = w["plasma"]
    cE, cB = C.solver_coefficients(w["solver"], dt, w["dz"])
    o = oracle.Oracle(nz_sample, w["nr"], w["n_modes"], w["dz"], w["dr"], dt, cE, cB,
                      C.filter_taps(cB), periodic=True,
                      partitions=4 * threads if threads > 1 else 1, threads=threads)
    # the slab sits on the plateau of the profile (z_start + ramp onwards)
    first = int(np.ceil((pl["z_start"] + pl["ramp_len"]) / w["dz"]))
    p = S.plasma_cells(np.arange(first, first + nz_sample), w["nr"], w["dz"], w["dr"],
                       pl["n0"], pl["z_start"], pl["ramp_len"], pl["ppc"], pl["seed"])
    p["z"] = p["z"] - first * w["dz"]
    o.load_particles(**p)
    n = o.num_particles()
    t0 = time.perf_counter()
    o.step(steps)
    t = time.perf_counter() - t0
    return n * steps / t, n, t


# Arm (implementer 0x41) part numbers that /proc/cpuinfo gives in place of a model name
_ARM_PARTS = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1",
              "0xd49": "Arm Neoverse N2", "0xd84": "Arm Neoverse V3"}


def _host_cpu():
    """CPU model and core count of this host (for the CPU baseline's record)"""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            k, _, v = line.partition(":")
            if k.strip() in ("model name", "Model Name", "CPU part") and v.strip():
                model = v.strip()
                if k.strip() == "CPU part":
                    model = _ARM_PARTS.get(model.lower(), "Arm part " + model)
                break
    except OSError:
        pass
    import platform
    return {"model": model or platform.processor() or platform.machine(), "cpus": os.cpu_count()}


def _config(args, w, ws):
    """the workload keys both arms report"""
    return {"workload": args.workload, "nz": w["nz"], "nr": w["nr"], "modes": w["n_modes"],
            "ppc": list(w["plasma"]["ppc"]), "solver": "dual L=16", "parallelism": "replicas x%d" % ws}


def run_reference(args, w):
    """--impl reference: the FP64 CPU oracle (this repository's reference
    implementation of the method) on the host cores, bounded per step."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import coeffs as C
    dt = 0.9 * C.cfl_dt(w["dz"], w["dr"], w["nr"], w["n_modes"], w["solver"])
    nz_s = args.ref_nz
    import oracle
    nth = (os.cpu_count() or 1) if oracle.Oracle.has_openmp() else 1
    oracle_sample(w, dt, nz_s, max(1, args.warmup), threads=nth)      # warm-up (untimed)
    rate, n, t = oracle_sample(w, dt, nz_s, args.steps, threads=nth)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "particle-steps/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(_config(args, w, ws), dt=dt,
                       sample="each step: a periodic z-slab of %d of the %d columns (%d particles)"
                              % (nz_s, w["nz"], n)),
        "cpu_baseline": {"value": rate, "unit": "particle-steps/s", "cores": nth, "kind": "oracle",
                         "sample": "%d steps of a %d x %d periodic slab (%d particles)%s"
                                   % (args.steps, nz_s, w["nr"], n,
                                      ", OpenMP over %d particle ranges" % (4 * nth) if nth > 1 else "")},
        "e2e": {"value": rate, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def aggregate_ranks(ms, particles, steps, ws, device):
    """Whole-job throughput over ranks: the slowest rank's time (max) and all
    ranks' particles (sum).  Returns (ms_max, particles_all, particle-steps/s)."""
    import torch
    ms_t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    tot_p = torch.tensor([float(particles)], device=device, dtype=torch.float64)
    if ws > 1:
        torch.distributed.all_reduce(ms_t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(tot_p)
    ms_max = float(ms_t.item())
    particles_all = float(tot_p.item())
    return ms_max, particles_all, particles_all * steps / (ms_max / 1e3)


def run_ours(args, w):
    import torch
    import paper_2303_12874_gb300 as q
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    sim = _make_sim(q, w, stream)
    _init_state(sim, w)
    for _ in range(args.warmup):
        sim.step(1)
    n0 = sim.diag()["particles"]

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- timed region: K full steps, CUDA events on the library's stream
    launches0 = sim.launch_count()
    clocks = ClockSampler(dev)
    barrier()
    if rank == 0:
        clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    barrier()
    clk = clocks.stop() if rank == 0 else None
    launches = sim.launch_count() - launches0
    n1 = sim.diag()["particles"]
    n_avg = 0.5 * (n0 + n1)
    ms_max, particles_all, value = aggregate_ranks(ms, n_avg, args.steps, ws, "cuda")
    cells = w["nz"] * w["nr"]
    cell_updates = ws * cells * args.steps / (ms_max / 1e3)

    # ---- per-kernel times: a second run of the same kind of steps with CUDA
    # events around every kernel class.  Its launches are queued behind a GPU
    # sleep, so no host delay falls between a pair of events; the per-class
    # times then add up to no more than the pass itself.
    sim.profile(True, True)
    torch.cuda._sleep(int(2e8))
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    sim.step(args.prof_steps)
    p1.record(stream)
    torch.cuda.synchronize()
    prof_total_ms = p0.elapsed_time(p1)
    kt = sim.kernel_times()
    sim.profile(False, True)
    dt_used = sim.dt
    gpd_ms, gpd_n = kt["gather_push_deposit"]
    gpd_avg = gpd_ms / max(gpd_n, 1)
    solver_ms = sum(kt[k][0] for k in ("faraday", "j_decode", "jz_filter", "ampere"))
    ppc = int(np.prod(w["plasma"]["ppc"]))
    gpd_bytes = n_avg * (GPD_BYTES_PER_PARTICLE + GPD_BYTES_PER_CELL / ppc)
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured"
    if not hbm:
        hbm, peak_src = 6800.0, "fallback"
    achieved = gpd_bytes / (gpd_avg / 1e3) / 1e9
    traffic = _measured_traffic(args.workload, q.KERNEL_REV)
    nkeys = -(-w["nz"] // 16) * 16 * (-(-w["nr"] // 8) * 8)     # sort keys: cells rounded up to whole tiles
    kernels = {}
    for k, (kms, kn) in kt.items():
        if not kn:
            continue
        b = kernel_bytes(k, w, n_avg, kn, nkeys)
        ent = {"ms_per_step": kms / max(args.prof_steps, 1), "launches": int(kn)}
        if b is not None and kms > 0:
            gbs = b / (kms / 1e3) / 1e9
            ent.update({"algorithmic_bytes_per_launch": b / kn, "achieved_gbs": gbs,
                        "frac_of_measured_hbm": gbs / hbm})
        kernels[k] = ent
    # ---- end to end through the C ABI with host buffers (rank-local)
    e2e = None
    if not args.no_e2e:
        p = sim.particles()
        pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy() for k, v in p.items()}
        out_n = len(pin["z"])
        # the final particles come back into pinned memory too (headroom for injection)
        pout = torch.empty(9 * (out_n + out_n // 4 + 4096), dtype=torch.float64).pin_memory().numpy()
        nsteps_e2e = args.e2e_steps if args.e2e_steps > 0 else args.steps
        sim2 = _make_sim(q, w, stream)
        fields_h = {}          # (re, im) per field in pinned host memory
        for which in ("E", "B"):
            for c in ("r", "phi", "z"):
                for m in range(w["n_modes"]):
                    f = sim.get_field(which, c, m)
                    fields_h[(which, c, m)] = tuple(
                        torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy() for x in (f.real, f.imag))
        torch.cuda.synchronize()
        # each phase ends with a read back to the host or a synchronous copy,
        # so the marks between them add no waits
        t0 = time.perf_counter()
        sim2.load_particles(pin["z"], pin["r"], pin["phi"], pin["ux"], pin["uy"], pin["uz"], pin["w"])
        t1 = time.perf_counter()
        for (which, c, m), v in fields_h.items():
            sim2.set_field(which, c, m, v)
        t2 = time.perf_counter()
        for _ in range(nsteps_e2e):
            sim2.step(1)
            d = sim2.diag()
        t3 = time.perf_counter()
        res = sim2.particles(out=pout)
        t = time.perf_counter() - t0
        phases = {"load_particles": t1 - t0, "set_fields": t2 - t1, "steps_and_diag": t3 - t2,
                  "particles_out": t0 + t - t3}
        h2d = out_n * 7 * 8 + sum(re.size * 16 for re, _ in fields_h.values())
        d2h = len(res["z"]) * 9 * 8 + nsteps_e2e * (7 + w["n_modes"]) * 8
        e2e = {"value": ws * out_n * nsteps_e2e / t, "unit": "particle-steps/s",
               "h2d_bytes_per_step": int(h2d / nsteps_e2e),
               "d2h_bytes_per_step": int(d2h / nsteps_e2e),
               "steps": nsteps_e2e, "phases_s": {k: round(v, 4) for k, v in phases.items()},
               "note": "state loaded from pinned host memory once, "
               "diagnostics read back every step, final particles read back into pinned memory"}
        sim2.close()
        del d

    # ---- the FP32 float-atomic deposit variant on the same workload and GPU
    fatomic = None
    if not args.no_fatomic:
        sim.close()
        sfa = _make_sim(q, w, stream, precision=q.QPIC_FP32_FATOMIC)
        _init_state(sfa, w)
        sfa.step(args.warmup)
        nfa = sfa.diag()["particles"]
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        sfa.step(args.fatomic_steps)
        g1.record(stream)
        torch.cuda.synchronize()
        msfa = g0.elapsed_time(g1)
        sfa.profile(True, True)
        sfa.step(2)
        kfa = sfa.kernel_times()
        sfa.profile(False, False)
        gfa = kfa["gather_push_deposit"]
        fatomic = {"value": nfa * args.fatomic_steps / (msfa / 1e3), "unit": "particle-steps/s",
                   "cell_updates_per_s": w["nz"] * w["nr"] * args.fatomic_steps / (msfa / 1e3),
                   "ms_per_step": msfa / args.fatomic_steps, "steps": args.fatomic_steps,
                   "gpd_ms": gfa[0] / max(gfa[1], 1), "dtype": "f32",
                   "note": "same kernels, current summed by FP32 float atomics in global memory"}
        sfa.close()

    # ---- per-particle work in the directional split (Eq. 17) on the same workload
    work = None
    if not args.no_work:
        sim.close()
        swk = _make_sim(q, w, stream, track_work=2)
        _init_state(swk, w)
        swk.step(args.warmup)
        nwk = swk.diag()["particles"]
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        swk.step(args.work_steps)
        g1.record(stream)
        torch.cuda.synchronize()
        mswk = g0.elapsed_time(g1)
        swk.profile(True, True)
        swk.step(2)
        kwk = swk.kernel_times()
        swk.profile(False, False)
        gwk = kwk["gather_push_deposit"]
        work = {"value": nwk * args.work_steps / (mswk / 1e3), "unit": "particle-steps/s",
                "ms_per_step": mswk / args.work_steps, "steps": args.work_steps,
                "gpd_ms": gwk[0] / max(gwk[1], 1), "dtype": "f32",
                "note": "track_work = 2: W_z and W_perp per particle (Eq. 17), 8 B more read "
                        "and written per particle-step"}
        swk.close()

    # ---- the reduced model of Eq. 8 (FP64 Dormand-Prince, one thread per electron)
    reduced = None
    if not args.no_reduced:
        try:
            reduced = reduced_leg(q, torch, stream, args)
        except Exception as e:                          # an auxiliary leg never voids the main line
            reduced = {"error": "%s: %s" % (type(e).__name__, e)}

    # ---- the plain FP64 GPU path on the same workload and GPU
    fp64 = None
    if not args.no_fp64:
        sim.close()
        s64 = _make_sim(q, w, stream, precision=q.QPIC_FP64)
        _init_state(s64, w)
        for _ in range(2):
            s64.step(1)
        n64 = s64.diag()["particles"]
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s64.step(args.fp64_steps)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        fp64 = {"value": n64 * args.fp64_steps / (ms64 / 1e3), "unit": "particle-steps/s",
                "cell_updates_per_s": w["nz"] * w["nr"] * args.fp64_steps / (ms64 / 1e3),
                "ms_per_step": ms64 / args.fp64_steps, "steps": args.fp64_steps,
                "dtype": "f64", "note": "one thread per particle, FP64 atomics, no tiles or sort"}
        s64.close()

    # ---- optional: batched parameter scan (independent runs, one graph launch per cycle)
    batch = None
    if args.batch_runs > 0:
        batch = batch_scan(q, torch, stream, args.batch_runs, args.batch_steps)

    # ---- CPU baseline: the oracle as it stands on a bounded sample (rank 0, N = 1)
    cpu = None
    cpu_all = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        rate, n, t = oracle_sample(w, dt_used, args.ref_nz, args.cpu_steps)
        cpu = {"value": rate, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
               "sample": "%d steps of a %d x %d periodic z-slab of the workload (%d particles), "
                         "single-threaded FP64 C, %.1f s" % (args.cpu_steps, args.ref_nz, w["nr"], n, t),
               "host": _host_cpu()}
        nth = os.cpu_count() or 1
        if nth > 1:
            import oracle
            if oracle.Oracle.has_openmp():
                steps_all = max(args.cpu_steps, 4 * args.cpu_steps * min(nth, 16) // 16)
                rate, n, t = oracle_sample(w, dt_used, args.ref_nz, steps_all, threads=nth)
                cpu_all = {"value": rate, "unit": "particle-steps/s", "cores": nth, "kind": "oracle",
                           "sample": "%d steps of the same slab (%d particles), FP64 C with OpenMP over "
                                     "%d particle ranges, %.1f s" % (steps_all, n, 4 * nth, t)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": dict(_config(args, w, ws), particles_per_gpu=int(n_avg), dt=dt_used,
                           deposit="int64 fixed point",
                           l2="inputs larger than L2 (particles %.1f GB)" % (n_avg * 36 / 1e9)),
            "cell_updates_per_s": cell_updates,
            "solver_cell_updates_per_s": cells * args.prof_steps / (solver_ms / 1e3) if solver_ms else None,
            "gpd_particle_steps_per_s": n_avg / (gpd_avg / 1e3),
            "kernels": kernels,
            "kernel_pass": {"steps": args.prof_steps, "ms_per_step": prof_total_ms / max(args.prof_steps, 1),
                            "kernels_ms_per_step_sum": sum(v["ms_per_step"] for v in kernels.values()),
                            "note": "per-kernel times from CUDA events in a second pass of the same steps, "
                                    "its launches queued behind a GPU sleep"},
            "roofline": {"kernel": "gather_push_deposit", "bound": "hbm", "achieved": achieved,
                         "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "peak_source": peak_src + " (hbm_gbs, burst)",
                         "algorithmic_bytes_per_launch": gpd_bytes, "traffic": traffic},
            "fp64_gpu_path": fp64,
            "fp32_float_atomic_path": fatomic, "work_tracking_path": work, "reduced_model_path": reduced,
            "batch_scan": batch,
            "fp32_over_fp64": (value / ws / fp64["value"]) if fp64 else None,
            "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches,
        }
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg2_lwfa")
    ap.add_argument("--prof-steps", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="steps of the end-to-end leg (0: the same as --steps)")
    ap.add_argument("--ref-nz", type=int, default=100)
    ap.add_argument("--no-fatomic", action="store_true")
    ap.add_argument("--no-work", action="store_true")
    ap.add_argument("--no-reduced", action="store_true")
    ap.add_argument("--reduced-electrons", type=int, default=1 << 20)
    ap.add_argument("--reduced-steps", type=int, default=200)
    ap.add_argument("--reduced-divergence-electrons", type=int, default=1 << 16,
                    help="electrons of the staggering-factor comparison (0: skip it)")
    ap.add_argument("--work-steps", type=int, default=20)
    ap.add_argument("--fatomic-steps", type=int, default=20)
    ap.add_argument("--cpu-steps", type=int, default=24,
                    help="oracle steps timed for cpu_baseline (about 10 s on one core)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--batch-runs", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=500)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    w = synth.workload(args.workload)
    if args.impl == "reference":
        return run_reference(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
