"""Benchmark of the multi-state QHFPE hot path on GB300.

Workload: the two-state photoisomerization model (quartic double-well ground state, displaced
anharmonic excited state, constant diabatic coupling 0.5) on a 96 x 128 (q x p) grid, Drude bath
eta = 1, gamma = 1, beta = 1 with two Matsubara terms and the delta-term, hierarchy depth 8 (165
elements x 4 electronic pairs = 8.11 M phase-space cells).  One step = one RK4 step of every cell of
the whole hierarchy (four right-hand-side stages: upwind kinetic stencil, FFT potential kernel with
diabatic mixing, bath and tier couplings, Horner update) plus the FP64 trace Tr{mu W^(0)} that the
response functions record.  Metric: phase-space cell-updates per second.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead (bounded sample).
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

METRIC = "phase-space cell-updates/s"
L2_BYTES = 129 * 2 ** 20


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest of `value` over all ranks (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, steps, world, max_ms):
    """Whole-job units per second: every rank processes its own replicas (no shared work)."""
    return units_per_rank * steps * world / (max_ms / 1e3)


def workload():
    import qhfpe_inputs as qi
    m = qi.photoisomerization_two_state()
    return m, qi.u_table(m)


def cells_of(m, n_elem):
    return n_elem * m["S"] * m["S"] * m["nq"] * m["np"]


class Clocks:
    """SM clock, power and clock-event (throttle) reasons of THIS process's GPU, sampled every ~2 ms
    while the benchmark runs; samples taken while the timed region is open are kept apart.

    The GPU is named by its UUID (from torch), never by an index: nvidia-smi and NVML do not see
    CUDA_VISIBLE_DEVICES, so an index can name another user's GPU.  Queries are read-only: in-process
    NVML through ctypes when the driver library loads, else `nvidia-smi -i GPU-<uuid>` at 20 ms."""

    # clock-event reason bits of NVML
    BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
            0x80: "hw_power_brake_slowdown"}
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, local_index):
        import torch
        self.uuid = None
        try:
            u = str(torch.cuda.get_device_properties(local_index).uuid)
            self.uuid = u if u.startswith("GPU-") else "GPU-" + u
        except (AttributeError, RuntimeError):
            pass
        self.rows = []          # (sm_mhz, reasons bitmask or names, power_w, in_timed)
        self.max_mhz = None
        self.timed = False
        self.source = None
        self.error = None
        self._stop = threading.Event()
        self._nvml = None
        self.proc = None
        self.t = None

    # -- NVML through ctypes ------------------------------------------------------------------------
    def _nvml_open(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit_v2 failed")
        h = ctypes.c_void_p()
        if lib.nvmlDeviceGetHandleByUUID(self.uuid.encode(), ctypes.byref(h)) != 0:
            raise OSError("no NVML device with UUID " + self.uuid)
        mx = ctypes.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:  # NVML_CLOCK_SM
            self.max_mhz = float(mx.value)
        reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self._nvml = (ctypes, lib, h, reasons)

    def _nvml_loop(self):
        ctypes, lib, h, reasons = self._nvml
        clk, pw, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            ok = lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0
            r = reasons(h, ctypes.byref(rs)) == 0
            p = lib.nvmlDeviceGetPowerUsage(h, ctypes.byref(pw)) == 0
            if ok:
                self.rows.append((float(clk.value), int(rs.value) if r else 0, pw.value / 1e3 if p else None,
                                  self.timed))
            self._stop.wait(0.002)

    # -- nvidia-smi fallback ------------------------------------------------------------------------
    def _smi_loop(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7 or not parts[0].replace(".", "").isdigit():
                continue
            if parts[1].replace(".", "").isdigit():
                self.max_mhz = float(parts[1])
            act = [names[k] for k in range(4) if parts[3 + k].lower() == "active"]
            pw = float(parts[2]) if parts[2].replace(".", "").isdigit() else None
            self.rows.append((float(parts[0]), act, pw, self.timed))

    def __enter__(self):
        if self.uuid is None:
            self.error = "no device UUID from torch"
            return self
        try:
            self._nvml_open()
            self.source = "nvml (in-process, read-only, ~2 ms)"
            self.t = threading.Thread(target=self._nvml_loop, daemon=True)
        except (OSError, AttributeError) as ex:
            self.error = f"nvml: {ex}"
            try:
                self.proc = subprocess.Popen(["nvidia-smi", "-i", self.uuid, f"--query-gpu={self.Q}",
                                              "--format=csv,noheader,nounits", "-lms", "20"],
                                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                self.source = "nvidia-smi -i <uuid> -lms 20"
                self.t = threading.Thread(target=self._smi_loop, daemon=True)
            except OSError as ex2:
                self.error += f"; nvidia-smi: {ex2}"
                return self
        self.t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        if self._nvml:
            self._nvml[1].nvmlShutdown()

    def _names(self, r):
        if isinstance(r, list):
            return set(r)
        return {n for b, n in self.BITS.items() if r & b}

    def summary(self):
        timed = [r for r in self.rows if r[3]]
        use = timed if timed else self.rows
        out = {"sm_mhz": statistics.median(r[0] for r in use) if use else None, "sm_max_mhz": self.max_mhz,
               "reasons": sorted(set().union(*[self._names(r[1]) for r in use])) if use else ["unsampled"],
               "samples_timed": len(timed), "samples_total": len(self.rows), "source": self.source,
               "gpu_uuid": self.uuid}
        pw = [r[2] for r in use if r[2] is not None]
        if pw:
            out["power_w_max"] = max(pw)
        if not timed:
            out["note"] = "no sample inside the timed region; figures from the whole run" if use else \
                (self.error or "no samples")
        return out


SPEC2D = dict(n_t1=64, t1_stride=8, t2=[0, 100, 200, 300], n_t3=512)
# FP64 stage kernel on the benchmark workload: (2 DFMA + DADD + DMUL) per cell per stage, ncu count of
# the current kernel (the p-diagonal bath terms in the r-space mixing)
FP64_FLOPS_PER_CELL_STAGE = (2 * 348410880 + 287308800 + 61332480) / 8110080
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12


def spectrum_2d_measure(stream):
    """Batched 2D electronic spectrum on the two-state harmonic model (32 x 32, depth 3, dt 0.01):
    64 coherence delays (stride 8 steps) x 4 waiting times x 2 first-interaction pathways = 512
    detection propagations of 512 steps, packed as replicas of one batch per phase and replayed from
    captured graphs.  Wall time of the whole schedule (equilibrium given) for the mixed and the FP64
    form; the mixed form's relative L2 error against the FP64 form on R3 and on the correlation spectra
    (the FP64 form itself matches the CPU oracle to 1e-10 in the parity tests)."""
    import numpy as np
    import torch
    import qhfpe_inputs as qi
    from paper_1706_09590_gb300 import Propagator
    m = qi.harmonic_two_state()
    T = qi.u_table(m)
    eqp = Propagator(m, T, precision="fp64", stream=stream)
    eqp.equilibrate(3000)
    W_eq = eqp.get_state(0)
    eqp.close()
    out = {}
    R = {}
    args = (SPEC2D["n_t1"], SPEC2D["t1_stride"], SPEC2D["t2"], SPEC2D["n_t3"])
    for prec in ("mixed", "fp64"):
        P = Propagator(m, T, precision=prec, stream=stream)
        P.set_equilibrium(W_eq)
        P.third_order_response(*args, split_pathways=True)  # builds the batches and graphs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        R[prec] = P.third_order_response(*args, split_pathways=True)
        torch.cuda.synchronize()
        out[prec + "_s"] = time.perf_counter() - t0
        if prec == "mixed":
            # the same schedule with every phase's propagation as one persistent cooperative launch
            P.set_persistent(True)
            P.third_order_response(*args, split_pathways=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Rp = P.third_order_response(*args, split_pathways=True)
            torch.cuda.synchronize()
            out["mixed_persistent_s"] = time.perf_counter() - t0
            out["rel_err_R3_persistent_vs_graphs"] = float(np.linalg.norm(Rp - R[prec]) / np.linalg.norm(R[prec]))
            P.set_persistent(False)
        if prec == "mixed":
            w = np.linspace(5.0, 16.0, 111)
            spec = {}
            for b in range(len(SPEC2D["t2"])):
                full = R[prec][0, b] + R[prec][1, b]
                spec[b] = P.spectrum_2d(full, SPEC2D["t1_stride"] * m["dt"], m["dt"], w, w)[2]
            out["_spec_mixed"] = spec
            out["_w"] = w
        else:
            errs = []
            for b in range(len(SPEC2D["t2"])):
                full = R[prec][0, b] + R[prec][1, b]
                ref = P.spectrum_2d(full, SPEC2D["t1_stride"] * m["dt"], m["dt"], out["_w"], out["_w"])[2]
                got = out["_spec_mixed"][b]
                errs.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
            out["rel_err_corr_spectra_vs_fp64"] = max(errs)
        P.close()
    a, b = R["mixed"], R["fp64"]
    out["rel_err_R3_vs_fp64"] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    out.pop("_spec_mixed")
    out.pop("_w")
    cells = 4 * 4 * 32 * 32
    out["workload"] = ("harmonic_32x32_d3, 64 t1 x 4 t2 x 2 pathways = 512 t3 jobs of 512 steps "
                       f"({512 * cells} cells per detection stage)")
    out["t3_cell_updates"] = 512 * cells * SPEC2D["n_t3"]
    return out


def linear_absorption_measure(stream):
    """Linear absorption of the two-state harmonic model (32 x 32, depth 3, terminator, dt 0.01, 2000 RK4
    steps of one 16,384-cell propagation): wall time of R1 with graph-replayed stage launches and with one
    persistent cooperative launch (FP64 and mixed), and the mixed form's R1 error against FP64."""
    import numpy as np
    import torch
    import qhfpe_inputs as qi
    from paper_1706_09590_gb300 import Propagator
    m = qi.harmonic_two_state()
    T = qi.u_table(m)
    E = Propagator(m, T, precision="fp64", stream=stream)
    E.equilibrate(1000)
    Weq = E.get_state(0)
    E.close()
    out = {"workload": "harmonic_32x32_d3, R1 over 2000 RK4 steps (one propagation, 16384 cells)"}
    R = {}
    for prec in ("fp64", "mixed"):
        for persistent in (False, True):
            P = Propagator(m, T, precision=prec, stream=stream)
            P.set_persistent(persistent)
            P.set_equilibrium(Weq)
            P.linear_response(2000)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            R[(prec, persistent)] = P.linear_response(2000)
            torch.cuda.synchronize()
            out[prec + ("_persistent_s" if persistent else "_graphs_s")] = time.perf_counter() - t0
            P.close()
    ref = R[("fp64", False)]
    out["rel_err_R1_mixed_vs_fp64"] = float(np.linalg.norm(R[("mixed", False)] - ref) / np.linalg.norm(ref))
    out["rel_err_R1_persistent_vs_graphs_fp64"] = float(np.linalg.norm(R[("fp64", True)] - ref) / np.linalg.norm(ref))
    return out


def learned_closure_measure(stream):
    """Learned closures on the two-state harmonic model at 96 x 128 (q, p in [-8, 8)): trained on depth-12 FP64 runs
    at eta in {0.2, 0.5, 1}, deployed at depth 4, judged at the held-out eta = 0.3 against depth 12: R1
    over 10 time units for the truncation, the Eq. (GMFP) terminator, the coefficient form (QHFPE_LEARNED)
    and the state-input network (QHFPE_LEARNED_STATE); their training times (device kernels), the wall
    time of R1 at depth 4 and at depth 12, and the pathway-additivity defect of a small third-order
    schedule (ket + bra against the full commutator) of each form."""
    import numpy as np
    import torch
    import qhfpe_inputs as qi
    from paper_1706_09590_gb300 import Propagator
    from paper_1706_09590_gb300 import closure as pcl
    base = qi.harmonic_two_state(nq=96, n_p=128, qr=(-8.0, 8.0), pr=(-8.0, 8.0), depth=12, eta=1.0)
    T = qi.u_table(base)
    probe = Propagator(base, T, precision="fp64", stream=stream)
    dt = 0.8 * probe.max_stable_dt()
    probe.close()
    base["dt"] = dt
    etas = (0.2, 0.5, 1.0)
    args = dict(deep_depth=12, target_tier=5, n_eq=int(10 / dt), n_prop=int(6 / dt), every=max(1, int(0.2 / dt)))
    out = {"workload": "harmonic two-state 96x128, depth 12 -> 4, train eta 0.2/0.5/1, judged at eta 0.3, R1 over 10 "
                       "time units", "dt": dt}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Xc, Sc = pcl.training_set(base, T, etas, stream=stream, **args)
    out["coef_data_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    wc, _ = pcl.train(Xc, Sc, n_iters=3000, batch=4096, lr=1e-3)
    out["coef_train_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    Xs, Ys = pcl.state_training_set(base, T, etas, stream=stream, **dict(args, every=max(1, int(0.5 / dt))))
    out["state_data_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    ws, _ = pcl.train_state(2, Xs, Ys, n_iters=3000, batch=4096, lr=1e-3)
    out["state_train_s"] = time.perf_counter() - t0
    out["state_samples"] = int(Xs.shape[0])
    n_t = int(10 / dt)
    R1, defect = {}, {}
    for name, depth, closure in (("depth12", 12, 1), ("truncate", 4, 0), ("terminator", 4, 1), ("learned_coef", 4, 2),
                                 ("learned_state", 4, 3)):
        m = dict(base, eta=0.3, depth=depth, closure=closure)
        P = Propagator(m, T, precision="fp64", stream=stream)
        if closure == 2:
            P.closure_load(wc)
        if closure == 3:
            P.closure_state_load(ws)
        P.equilibrate(int(10 / dt))
        P.set_equilibrium(P.get_state(0))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        R1[name] = P.linear_response(n_t)
        torch.cuda.synchronize()
        out[name + "_R1_s"] = time.perf_counter() - t0
        sched = (2, int(0.5 / dt), [0, int(1.0 / dt)], int(2 / dt))
        full = P.third_order_response(*sched)
        split = P.third_order_response(*sched, split_pathways=True)
        defect[name] = float(np.linalg.norm(split[0] + split[1] - full) / np.linalg.norm(full))
        P.close()
    ref = R1["depth12"]
    out["rel_err_R1_vs_depth12"] = {k: float(np.linalg.norm(v - ref) / np.linalg.norm(ref)) for k, v in R1.items()
                                    if k != "depth12"}
    out["additivity_defect"] = defect
    return out


def cpu_spectrum_baseline(seconds_cap=60.0):
    """The FP64 oracle as it stands on this host's cores, on a bounded sub-schedule of the batched 2D
    spectrum (ket pathway, the first two t1 delays, the first two waiting times, full t3 = 512 steps),
    extrapolated to the full schedule by the number of RK4 steps (every step of the schedule costs
    the same: one full-hierarchy step of the 32 x 32, depth-3 model)."""
    import oracle
    import qhfpe_inputs as qi
    m = qi.harmonic_two_state()
    O = oracle.Oracle(m)
    W_eq, _ = O.equilibrate(300)
    n_t1, t2, n_t3, stride = 2, SPEC2D["t2"][:2], SPEC2D["n_t3"], SPEC2D["t1_stride"]
    t0 = time.perf_counter()
    O.third_order_response(W_eq, n_t1, stride, t2, n_t3, first=oracle.LEFT)
    dt = time.perf_counter() - t0

    def steps(n1, t2s, n3):  # RK4 steps of one pathway
        return (n1 - 1) * stride + n1 * (max(t2s) + len(t2s) * n3)
    full = 2 * steps(SPEC2D["n_t1"], SPEC2D["t2"], n_t3)
    sample = steps(n_t1, t2, n_t3)
    return {"sample_s": dt, "sample": f"ket pathway, {n_t1} t1 x {len(t2)} t2 x t3 {n_t3} ({sample} RK4 steps)",
            "full_schedule_steps": full, "extrapolated_s": dt * full / sample, "cores": oracle.num_threads(),
            "kind": "oracle"}


def paper_workload_measure(stream):
    """The paper's own model (Sec. III: Morse diabats, Gaussian coupling, 512 x 128 mesh, underdamped
    bath at depth 5; 1.57 M cells, L2-resident): RK4 throughput of the mixed form (CUDA events on the
    launching stream), the fused stage kernel's time per launch, and the linear absorption spectrum
    from the FP64 equilibrium in the mixed and FP64 forms (peak position in cm^-1 with omega_0 =
    100 cm^-1, the mixed form's relative L2 error on R1)."""
    import numpy as np
    import torch
    import qhfpe_inputs as qi
    from paper_1706_09590_gb300 import Propagator
    m = qi.morse_photoisomerization()
    T = qi.u_table(m)
    out = {"workload": "morse_512x128_d5 (paper Sec. III model, underdamped zeta 40 cm^-1, gamma 500 cm^-1, "
                       "beta 0.48, dt 1e-3 / omega_0)"}
    P = Propagator(m, T, precision="mixed", stream=stream)
    P.set_state(qi.random_state(m, seed=1706))
    P.step(20)
    cells = int(np.prod(P.shape))
    n = 2000
    s = torch.cuda.current_stream() if stream is None else stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    P.step(n)
    e1.record(s)
    torch.cuda.synchronize()
    out["cells"] = cells
    out["cell_updates_per_s"] = cells * n / (e0.elapsed_time(e1) / 1e3)
    P.kernel_timing(True)
    P.step(200)
    kt = P.kernel_timing_read()
    P.kernel_timing(False)
    out["stage_us_per_launch"] = 1e3 * kt["stage"][1] / max(kt["stage"][0], 1)
    P.close()
    E = Propagator(m, T, precision="fp64", stream=stream)
    E.equilibrate(1500)
    Weq = E.get_state(0)
    E.close()
    omega = np.linspace(100.0, 300.0, 401)
    R = {}
    for prec in ("mixed", "fp64"):
        Q = Propagator(m, T, precision=prec, stream=stream)
        Q.set_equilibrium(Weq)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        R[prec] = Q.linear_response(1500)
        torch.cuda.synchronize()
        out["linear_response_" + prec + "_s"] = time.perf_counter() - t0
        I = Q.spectrum_absorption(R[prec], m["dt"], omega)
        out["absorption_peak_" + prec + "_cm-1"] = float(100.0 * omega[np.argmax(I)])
        Q.close()
    out["rel_err_R1_mixed_vs_fp64"] = float(np.linalg.norm(R["mixed"] - R["fp64"]) / np.linalg.norm(R["fp64"]))
    return out


def hetero_batch_measure(stream):
    """Eight two-state harmonic models that differ in q grid, depth, closure, bath and dt (np = 32, two
    states, FP32 mixed form), advanced together as one heterogeneous batch (every Horner stage of all
    eight one launch) and one after another on their own: wall time of the same RK4 steps, inputs
    resident on the device."""
    import numpy as np
    import torch
    import qhfpe_inputs as qi
    from paper_1706_09590_gb300 import Batch, Propagator
    specs = [(32, 3, 1, 0.5, 0.010), (24, 5, 0, 0.3, 0.008), (40, 4, 1, 1.0, 0.010), (48, 2, 1, 0.2, 0.012),
             (32, 6, 0, 0.5, 0.009), (28, 3, 1, 2.0, 0.010), (36, 4, 1, 0.7, 0.011), (44, 5, 0, 0.4, 0.010)]
    models = [qi.harmonic_two_state(nq=nq, n_p=32, depth=d, closure=c, eta=eta, dt=dt) for nq, d, c, eta, dt in specs]

    def make():
        Ps = [Propagator(m, qi.u_table(m), precision="mixed", stream=stream) for m in models]
        for k, P in enumerate(Ps):
            P.set_state(qi.random_state(P.model, seed=500 + k, hermitian=True))
        return Ps

    n = 400
    Ps = make()
    B = Batch(Ps)
    B.step(20)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B.step(n)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    tq = B.tile_rows()
    B.close()
    cells = sum(P.n_replicas * int(np.prod(P.shape)) for P in Ps)
    for P in Ps:
        P.close()
    Qs = make()
    for Q in Qs:
        Q.step(20)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for Q in Qs:
        Q.step(n)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    for Q in Qs:
        Q.close()
    return {"workload": "8 harmonic two-state models, np 32, nq 24-48, depth 2-6, terminator or truncation, "
                        f"eta 0.2-2, dt 0.008-0.012 ({cells} cells), {n} RK4 steps, FP32 mixed form",
            "batched_cell_updates_per_s": cells * n / t_batch, "one_by_one_cell_updates_per_s": cells * n / t_seq,
            "batched_s": t_batch, "one_by_one_s": t_seq, "tile_rows": tq, "timer": "wall clock, device synchronised"}


def three_state_measure(stream, hbm_peak):
    """The three-state workload at full size (256 x 256, depth 10, three bath modes: 286 elements x 9
    pairs, 168.7 M cells): RK4 throughput of the mixed and FP64 forms (CUDA events on the launching
    stream), the mixed fused stage kernel's time per launch and its fraction of the HBM peak on the
    algorithmic 22 B per cell per stage."""
    import numpy as np
    import torch
    import qhfpe_inputs as qi
    from paper_1706_09590_gb300 import Propagator
    m = qi.three_state()
    T = qi.u_table(m)
    W = qi.random_state(m, seed=1706)
    out = {"workload": "three_state_256x256_d10_K2 (3 states, 286 elements, 168.7 M cells)"}
    s = torch.cuda.current_stream() if stream is None else stream
    for prec, n in (("mixed", 20), ("fp64", 2)):
        P = Propagator(m, T, precision=prec, stream=stream)
        P.set_state(W)
        P.step(2)
        cells = int(np.prod(P.shape))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        P.step(n)
        e1.record(s)
        torch.cuda.synchronize()
        out[prec + "_cell_updates_per_s"] = cells * n / (e0.elapsed_time(e1) / 1e3)
        if prec == "mixed":
            P.kernel_timing(True)
            P.step(2)
            kt = P.kernel_timing_read()
            P.kernel_timing(False)
            ms = kt["stage"][1] / max(kt["stage"][0], 1)
            out["stage_ms_per_launch"] = ms
            out["stage_hbm_frac_of_measured"] = 22.0 * cells / (ms / 1e3) / 1e9 / hbm_peak
            out["tile_rows_autotuned"] = P.tile_rows()
        out["cells"] = cells
        P.close()
    return out


def tensor_core_measure(stream, m, T, tc_peak, peak_source):
    """The tensor-core form (tcgen05 split-bf16 DFT-GEMM potential term + fused stencil/bath kernel) on
    the benchmark workload: RK4 throughput (CUDA events on the launching stream) and the roofline of
    its potential kernel against the bf16 tensor peak, on the tensor flops it issues (forward and
    inverse DFT-GEMMs: 4 real products of [1 x np] x [np x np] per row, 3 bf16 products each)."""
    import numpy as np
    import torch
    import qhfpe_inputs as qi
    from paper_1706_09590_gb300 import Propagator
    P = Propagator(m, T, precision="bf16x3", stream=stream)
    P.set_state(qi.random_state(m, seed=1706))
    P.step(4)
    cells = int(np.prod(P.shape))
    s = torch.cuda.current_stream() if stream is None else stream
    n = 100
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    P.step(n)
    e1.record(s)
    torch.cuda.synchronize()
    P.kernel_timing(True)
    P.step(n)
    kt = P.kernel_timing_read()
    P.kernel_timing(False)
    P.close()
    n_pot, ms_pot = kt["potential"]
    n_stage, ms_stage = kt["stage"]
    pot_ms = ms_pot / max(n_pot, 1)
    flops = 2 * 3 * 4 * 2 * m["np"] * m["np"] * (cells / m["np"])
    return {"workload": "photoiso_96x128_d8_K2, precision bf16x3", "cell_updates_per_s": cells * n / (e0.elapsed_time(e1) / 1e3),
            "roofline": {"bound": "tensor", "kernel": "pot_tc_kernel (tcgen05 split-bf16 DFT-GEMM potential term)",
                         "achieved": flops / (pot_ms / 1e3) / 1e12, "peak": tc_peak, "unit": "TFLOP/s",
                         "frac": flops / (pot_ms / 1e3) / 1e12 / tc_peak, "peak_source": peak_source,
                         "ms_per_launch": pot_ms, "flops_per_launch": flops,
                         "share": ms_pot / max(ms_pot + ms_stage + kt["aux"][1], 1e-9)},
            "stage_ms_per_launch": ms_stage / max(n_stage, 1)}


def fp64_form_measure(stream, m, T, fp64_peak_tflops, peak_source):
    """The FP64 form on the benchmark workload: RK4 throughput and the fused stage kernel against the
    FP64 pipe (FP64 flops per launch as counted by ncu on this workload, FMA = 2)."""
    import numpy as np
    import torch
    import qhfpe_inputs as qi
    from paper_1706_09590_gb300 import Propagator
    P = Propagator(m, T, precision="fp64", stream=stream)
    P.set_state(qi.random_state(m, seed=1706))
    P.step(2)
    cells = int(np.prod(P.shape))
    s = torch.cuda.current_stream() if stream is None else stream
    n = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    P.step(n)
    e1.record(s)
    torch.cuda.synchronize()
    P.kernel_timing(True)
    P.step(4)
    kt = P.kernel_timing_read()
    P.kernel_timing(False)
    P.close()
    stage_ms = kt["stage"][1] / max(kt["stage"][0], 1)
    fl = FP64_FLOPS_PER_CELL_STAGE * cells
    return {"workload": "photoiso_96x128_d8_K2, precision fp64", "cell_updates_per_s": cells * n / (e0.elapsed_time(e1) / 1e3),
            "roofline": {"bound": "alu", "kernel": "fused_stage_kernel<double> (FP64 pipe)",
                         "achieved": fl / (stage_ms / 1e3) / 1e12, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                         "frac": fl / (stage_ms / 1e3) / 1e12 / fp64_peak_tflops, "peak_source": peak_source,
                         "ms_per_launch": stage_ms, "flops_per_launch": fl}}


SWEEP_ETAS = (0.1, 1.0, 5.0)
SWEEP_COUPLINGS = (0.2, 0.5, 1.0, 2.0)


def eta_coupling_sweep_measure(stream):
    """The benchmark model over its stated parameter ranges (eta in {0.1, 1, 5} x diabatic coupling in
    {0.2, 0.5, 1, 2}, 96 x 128, depth 8, two Matsubara terms + delta-term, dt = 0.8 x the stability
    bound): linear response over one time unit and the transient-absorption response (t1 = 0, waiting
    times 0 and 0.25, detection over 0.5) from one FP64 equilibrium, in the FP64 and the mixed form;
    each form's wall time and the mixed form's relative L2 error against FP64."""
    import numpy as np
    import torch
    import qhfpe_inputs as qi
    from paper_1706_09590_gb300 import Propagator
    rows = []
    for eta in SWEEP_ETAS:
        for coupling in SWEEP_COUPLINGS:
            m = qi.photoisomerization_two_state(eta=eta, coupling=coupling)
            T = qi.u_table(m)
            E = Propagator(m, T, precision="fp64", stream=stream)
            dt = 0.8 * E.max_stable_dt()
            E.close()
            E = Propagator(m, T, precision="fp64", stream=stream, dt=dt)
            E.equilibrate(300)
            Weq = E.get_state(0)
            E.close()
            # at eta = 5 the truncated hierarchy has growing modes (about e^(10 t)): compared up to t = 0.5
            t_r1, t_T, t_t3 = (0.5, 0.125, 0.375) if eta >= 5 else (1.0, 0.25, 0.5)
            n_r1, t2, n_t3 = int(round(t_r1 / dt)), [0, int(round(t_T / dt))], int(round(t_t3 / dt))
            R1, R3, wall = {}, {}, {}
            for prec in ("fp64", "mixed"):
                P = Propagator(m, T, precision=prec, stream=stream, dt=dt)
                P.set_equilibrium(Weq)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                R1[prec] = P.linear_response(n_r1)
                R3[prec] = P.third_order_response(1, 1, t2, n_t3)
                torch.cuda.synchronize()
                wall[prec] = time.perf_counter() - t0
                P.close()
            rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
            rows.append({"eta": eta, "coupling": coupling, "dt": dt, "rel_err_R1": rel(R1["mixed"], R1["fp64"]),
                         "rel_err_TAS_R3": rel(R3["mixed"], R3["fp64"]), "fp64_s": wall["fp64"],
                         "mixed_s": wall["mixed"]})
    return {"workload": "photoiso_96x128_d8_K2 at eta x coupling, R1 (1 time unit) + TAS R3 (T = 0, 0.25; t3 0.5); "
                        "eta 5: R1 0.5, T = 0, 0.125, t3 0.375 (growing modes of the truncated hierarchy)",
            "cases": rows, "max_rel_err": max(max(r["rel_err_R1"], r["rel_err_TAS_R3"]) for r in rows),
            "fp64_s_total": sum(r["fp64_s"] for r in rows), "mixed_s_total": sum(r["mixed_s"] for r in rows)}


def cpu_baseline(m, T, seconds=15.0):
    """The FP64 oracle as it stands, on this host's cores, over a bounded number of RK4 steps of the
    same workload (full hierarchy, full grid)."""
    import oracle
    import qhfpe_inputs as qi
    O = oracle.Oracle(m, T)
    W = qi.random_state(m, seed=1706)
    n = 0
    t0 = time.perf_counter()
    while True:
        W, _ = O.step(W, 1)
        n += 1
        if time.perf_counter() - t0 > seconds or n >= 50:
            break
    dt = time.perf_counter() - t0
    cells = cells_of(m, O.n_elem)
    return {"value": cells * n / dt, "unit": METRIC, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n} RK4 steps of the full 96x128 depth-8 hierarchy ({cells} cells), FP64, {dt:.1f} s"}


def run_reference(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    from oracle import build as ob
    ob.build()
    m, T = workload()
    import oracle
    import qhfpe_inputs as qi
    O = oracle.Oracle(m, T)
    W = qi.random_state(m, seed=1706)
    # bounded sample: W untimed steps (at most 3), then full RK4 steps of the whole workload until K
    # steps or about a minute of oracle time, so the run ends within a few minutes for any K and W
    n_warm = max(1, min(args.warmup, 3))
    W, _ = O.step(W, n_warm)
    t0 = time.perf_counter()
    done = 0
    while done < args.steps and (done == 0 or time.perf_counter() - t0 < 60.0):
        W, _ = O.step(W, 1)
        done += 1
    dt = time.perf_counter() - t0
    cells = cells_of(m, O.n_elem)
    val = cells * done / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "cell-updates/s", "n_gpus": args.gpus,
            "steps": done, "warmup": n_warm, "ms_per_step": 1e3 * dt / done,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "photoiso_96x128_d8_K2 (2 states, depth 8, 3 modes, 165 elements, "
                                   f"{cells} cells per GPU)", "precision": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": val, "unit": "cell-updates/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{done} timed RK4 steps of the full workload after {n_warm} warm-up "
                                       f"step(s) (of {args.steps} requested; capped at ~60 s of oracle time)"},
            "e2e": {"value": val, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed", "bf16x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-spectrum", action="store_true", help="skip the batched 2D-spectrum measurement")
    ap.add_argument("--no-paper-workload", action="store_true",
                    help="skip the measurement on the paper's own Morse model")
    ap.add_argument("--no-hetero-batch", action="store_true",
                    help="skip the heterogeneous-batch measurement")
    ap.add_argument("--no-three-state", action="store_true",
                    help="skip the full-size three-state measurement")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the tensor-core and FP64 forms on the benchmark workload")
    ap.add_argument("--no-closure", action="store_true",
                    help="skip the learned-closure measurement (two-state harmonic model, 96 x 128)")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the eta x coupling sweep of the benchmark model (FP64 vs mixed spectra)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1706_09590_gb300 import Propagator
    import qhfpe_inputs as qi

    m, T = workload()
    stream = torch.cuda.Stream()
    P = Propagator(m, T, precision=args.precision, stream=stream)
    cells = cells_of(m, P.n_elem)
    W0 = qi.random_state(m, seed=1706 + rank)
    P.set_state(W0)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident throughput --------------------------------------------------------------
    for _ in range(max(args.warmup, 3)):
        P.step(1, record_trace=True)
    barrier()
    P.kernel_timing(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        time.sleep(0.02)  # a few samples before the timed region
        barrier()
        clk.timed = True
        with torch.cuda.stream(stream):
            ev0.record(stream)
        tr = P.step(args.steps, record_trace=True)
        with torch.cuda.stream(stream):
            ev1.record(stream)
        barrier()
        clk.timed = False
    ms = ev0.elapsed_time(ev1)
    kt = P.kernel_timing_read()
    P.kernel_timing(False)
    ms = max_over_ranks(ms, dist, device="cuda")
    assert np.all(np.isfinite(tr)), "non-finite trace"
    value = job_throughput(cells, args.steps, world, ms)

    # ---- end to end through the C ABI with host buffers --------------------------------------------
    # every step: the state from pinned host memory, one RK4 step with its trace, the state back; the
    # mixed forms exchange complex64 states (their higher tiers are FP32 on the device), FP64 complex128
    n_e2e = max(2, min(args.steps, 10))
    if args.precision == "fp64":
        host_in = torch.from_numpy(W0.view(np.float64)).pin_memory()
        cdt = np.complex128
    else:
        host_in = torch.from_numpy(W0.astype(np.complex64).view(np.float32)).pin_memory()
        cdt = np.complex64
    host_out = torch.empty_like(host_in).pin_memory()
    w_in = host_in.numpy().view(cdt).reshape(P.shape)
    w_out = host_out.numpy().view(cdt).reshape(P.shape)
    state_bytes = host_in.numel() * host_in.element_size()
    barrier()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        P.set_state(w_in)
        P.step(1, record_trace=True)
        P.get_state(0, out=w_out)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, device="cuda")
    e2e = job_throughput(cells, n_e2e, world, 1e3 * e2e_s)

    # ---- roofline of the dominant kernel ------------------------------------------------------------
    import json as _j
    peaks = {}
    try:
        peaks = _j.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    tc_peak = peaks.get("bf16_tflops_sustained", 1700.0)
    tc_src = "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)" if "bf16_tflops_sustained" in peaks else \
        "fallback 1.7 PFLOP/s sustained"
    # FP64 peak: the DFMA rate measured on this device now (CUDA events; clocks as they are)
    from paper_1706_09590_gb300.qhfpe import fp64_fma_rate
    try:
        fp64_peak = fp64_fma_rate(stream, repeats=5) / 1e12
        fp64_src = "measured DFMA rate on this device (qhfpe_fp64_fma_rate, best of 5, of measured)"
    except RuntimeError:
        fp64_peak, fp64_src = FP64_PEAK_TFLOPS, "nominal FP64 rate (2 FMA / clock / SM, 152 SMs, 2.07 GHz)"
    n_stage, ms_stage = kt["stage"]
    n_pot, ms_pot = kt["potential"]
    esize = 8 if args.precision == "fp64" else 4
    # algorithmic bytes of one right-hand-side stage: the 11 state passes of a Horner RK4 step
    # (complex values) spread over its 4 stages
    alg_bytes_stage = 11 * 2 * esize * cells / 4
    stage_ms = ms_stage / max(n_stage, 1)
    pot_ms = ms_pot / max(n_pot, 1)
    total = max(ms_stage + ms_pot + kt["aux"][1], 1e-9)
    stage_name = "fused_window_kernel" if P.stage_form() == 1 else "fused_stage_kernel"
    stage_roof = {"bound": "hbm", "kernel": stage_name + " (FFT potential term, stencil, bath, tier couplings, "
                  "Horner update)" if args.precision != "bf16x3" else
                  "fused_stage_kernel (stencil, bath, tier couplings, Horner update; potential term read)",
                  "achieved": alg_bytes_stage / (stage_ms / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                  "frac": alg_bytes_stage / (stage_ms / 1e3) / 1e9 / hbm_peak, "traffic": None,
                  "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6800 GB/s",
                  "ms_per_launch": stage_ms, "share": ms_stage / total,
                  "algorithmic_bytes_per_launch": alg_bytes_stage}
    if args.precision == "fp64":
        # the FP64 form is bound by the FP64 pipe (ncu: 86 % of its cycles active, DRAM 3 %): FP64 flops
        # per launch (FMA = 2) as counted by ncu on this workload, against the DFMA rate measured here
        fl = FP64_FLOPS_PER_CELL_STAGE * cells
        stage_roof.update({"bound": "alu", "achieved": fl / (stage_ms / 1e3) / 1e12, "peak": fp64_peak,
                           "unit": "TFLOP/s", "frac": fl / (stage_ms / 1e3) / 1e12 / fp64_peak,
                           "peak_source": fp64_src, "flops_per_launch": fl})
        stage_roof.pop("algorithmic_bytes_per_launch")
    # DRAM bytes per launch from the committed ncu capture of the kernel this run times, valid only for
    # the kernel sources it was taken from
    try:
        import hashlib
        tr = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic_fused_window_photoiso_96x128_d8.json")))
        same = all(hashlib.sha256(open(os.path.join(ROOT, f), "rb").read()).hexdigest() == h
                   for f, h in zip(tr["sources"], tr["sources_sha256"]))
        if same and args.precision == "mixed" and P.stage_form() == 1:
            stage_roof["traffic"] = tr["dram_bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        pass
    roof = stage_roof
    if args.precision == "bf16x3" and n_pot:
        # tensor flops issued per launch: forward and inverse DFT-GEMMs, 4 real products of
        # [1 x np] x [np x np] per row, 3 bf16 products each
        flops = 2 * 3 * 4 * 2 * m["np"] * m["np"] * (cells / m["np"])
        tc_roof = {"bound": "tensor", "kernel": "pot_tc_kernel (tcgen05 split-bf16 DFT-GEMM potential term)",
                   "achieved": flops / (pot_ms / 1e3) / 1e12, "peak": tc_peak, "unit": "TFLOP/s",
                   "frac": flops / (pot_ms / 1e3) / 1e12 / tc_peak, "traffic": None,
                   "peak_source": tc_src, "ms_per_launch": pot_ms, "share": ms_pot / total,
                   "flops_per_launch": flops}
        roof = dict(tc_roof) if ms_pot >= ms_stage else dict(stage_roof)
        roof["other_kernel"] = stage_roof if ms_pot >= ms_stage else tc_roof

    line = {"metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"mixed": "f32", "bf16x3": "f32+bf16x3", "fp64": "f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": "photoiso_96x128_d8_K2 (2 states, depth 8, 3 modes, 165 elements, "
                                   f"{cells} cells per GPU)", "precision": args.precision,
                       "l2": f"working set {4 * cells * 2 * esize / 1e6:.0f} MB per step > 129 MB L2 (no flush)",
                       "tile_rows_autotuned": P.tile_rows(),
                       "stage_form_autotuned": {1: "q-window", 0: "general", -1: "none"}[P.stage_form()],
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": e2e, "unit": "cell-updates/s", "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes + 16 * 2},
            "gpu_launches": int(n_stage + n_pot + 2 * args.steps + 2),
            "roofline": roof, "clocks": clk.summary(),
            "fp64_peak": {"tflops": fp64_peak, "source": fp64_src}}
    walls = {}

    def timed(key, fn, *a):
        t0 = time.perf_counter()
        line[key] = fn(*a)
        walls[key] = round(time.perf_counter() - t0, 1)

    if args.precision == "mixed" and not args.no_forms:
        timed("tensor_core", tensor_core_measure, stream, m, T, tc_peak, tc_src)
        timed("fp64_form", fp64_form_measure, stream, m, T, fp64_peak, fp64_src)
    if not args.no_sweep:
        timed("eta_coupling_sweep", eta_coupling_sweep_measure, stream)
    if not args.no_closure:
        timed("learned_closure", learned_closure_measure, stream)
    if not args.no_spectrum:
        timed("linear_absorption", linear_absorption_measure, stream)
        timed("spectrum_2d", spectrum_2d_measure, stream)
        if not args.no_cpu_baseline and rank == 0:
            line["spectrum_2d"]["cpu_baseline"] = cpu_spectrum_baseline()
    if not args.no_paper_workload:
        timed("paper_workload", paper_workload_measure, stream)
    if not args.no_hetero_batch:
        timed("hetero_batch", hetero_batch_measure, stream)
    if not args.no_three_state:
        timed("three_state", three_state_measure, stream, hbm_peak)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        timed("cpu_baseline", cpu_baseline, m, T)
    line["section_wall_s"] = walls  # host wall time of each extra measurement, for the run's budget
    if rank == 0:
        print(json.dumps(line))
    P.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
