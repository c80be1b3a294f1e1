#!/usr/bin/env python3
"""Benchmark of the reverse-mode gradient path on one node; prints ONE JSON line.

Default workload: f(x) = ||A x||^2, A dense 10000 x 10000 FP64 (800 MB, larger
than L2), value-and-gradient through the C ABI (kg_grad), compared with the
forward pass alone (kg_eval): the paper's measure is the gradient/function
wall-clock ratio; the throughput is the gradient's algorithmic HBM bytes per
second.  Other workloads: --workload tet | dense32 | dense64 | laplace |
batched | autograd.

Multi-GPU (torchrun, one process per GPU): every rank runs an independent
replica of the workload (the problems are independent; there is no data-path
collective), timed between barriers; value = units of all ranks / max time.

--impl reference times the CPU oracle on the same workload, on rank 0 only:
the OpenMP build on all host cores for the dense and tet workloads (the full
problem per step), the serial oracle on a bounded sample for the others.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("gradient/function wall-clock ratio and gradient HBM GB/s (% of peak); "
          "batched grads/sec")
FALLBACK_HBM_GBS = 6800.0


# ------------------------------------------------------------------ peaks
def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    sm_mhz, sms = 2070.0, 152
    try:
        with open(path) as fh:
            P = json.load(fh)
        hbm, src = float(P["hbm_gbs"]), "measured"
        sm_mhz = float(P.get("sm_max_mhz", sm_mhz))
    except Exception:
        hbm, src = FALLBACK_HBM_GBS, "fallback"
    # FP64 FMA issue: 2 per SM per clock on GB300 (1.25 TFLOP/s nominal)
    fp64_tflops = sms * 2 * 2 * sm_mhz * 1e6 / 1e12
    # FP32 FMA issue: 128 per SM per clock
    fp32_tflops = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    return {"hbm_gbs": hbm, "hbm_src": src, "fp64_tflops": fp64_tflops,
            "fp32_tflops": fp32_tflops}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        # nvidia-smi numbers GPUs physically; a single visible device is named by
        # CUDA_VISIBLE_DEVICES when that is set
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        parts = [v for v in vis.split(",") if v.strip()]
        if parts and index < len(parts) and parts[index].strip().isdigit():
            index = int(parts[index])
        self.index = index
        self.proc = None
        self.path = None

    def wait_first_row(self, timeout_s: float = 5.0) -> bool:
        """Blocks until nvidia-smi has written its first sample (or timeout)."""
        t0 = time.perf_counter()
        while self.proc is not None and time.perf_counter() - t0 < timeout_s:
            self.fh.flush()
            try:
                if os.path.getsize(self.path) > 0:
                    return True
            except OSError:
                return False
            time.sleep(0.02)
        return False

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    power = float(parts[3]) if parts[3].replace(".", "", 1).isdigit() else None
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9], power))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        # the first sample may predate the load; the median is over the rest
        load = rows[1:] if len(rows) > 1 else rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, flags, _ in load for i, f in enumerate(flags)
                          if f.lower() == "active"})
        powers = [r[3] for r in load if r[3] is not None]
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(load),
                "power_w_max": max(powers) if powers else None}


def fp64_peak(peaks, box):
    """FP64 FMA peak for the ALU roofline: this run's kg_measure_box figure when
    it is there, else the nominal issue rate."""
    if box and box.get("fp64_fma_tflops", 0) > 0:
        return box["fp64_fma_tflops"], "measured in this run (kg_measure_box: FP64 FMA chains)"
    return peaks["fp64_tflops"], "nominal FP64 FMA issue rate: 152 SMs x 2 FMA/clk x 2070 MHz"


def cpu_baseline_runs(omp_fn, serial_fn, bytes_omp, what, budget_s, serial_bytes=None,
                      serial_what=None):
    """The CPU baseline: the OpenMP build of the oracle on all host cores (about
    60% of the budget), then the serial oracle (the rest).  Returns the
    cpu_baseline record: GB/s of algorithmic bytes, threads actually used, and
    the single-threaded figure beside it.  Without an OpenMP build, the serial
    oracle alone (cores 1)."""
    serial_bytes = bytes_omp if serial_bytes is None else serial_bytes
    serial_what = what if serial_what is None else serial_what

    def run(fn, nbytes, budget, cap):
        t0 = time.perf_counter()
        reps, out = 0, None
        while True:
            out = fn()
            reps += 1
            if time.perf_counter() - t0 >= budget or reps >= cap:
                break
        return reps * nbytes / 1e9 / (time.perf_counter() - t0), reps, out

    single = None
    try:
        v, reps, out = run(omp_fn, bytes_omp, 0.6 * budget_s, 400)
        cores = int(out[-1])
        rec = {"value": round(v, 4), "cores": cores,
               "sample": f"{reps} x {what} (oracle, OpenMP build, {cores} threads on the host cores)"}
        sb = 0.4 * budget_s
    except Exception as e:  # noqa: BLE001  (no OpenMP build on this host)
        rec, sb = None, budget_s
        single_note = f"OpenMP build unavailable: {e}"
    v1, reps1, _ = run(serial_fn, serial_bytes, sb, 20)
    single = {"value": round(v1, 4), "cores": 1,
              "sample": f"{reps1} x {serial_what} (oracle, 1 thread)"}
    if rec is None:
        return {**single, "kind": "oracle", "note": single_note}
    return {**rec, "kind": "oracle", "single_thread": single}


# ------------------------------------------------------------------ workloads
class Workload:
    """One value-and-gradient step of the path (`step`), its forward alone
    (`eval_step`), the same step through host buffers (`e2e_step`), byte /
    flop accounting and a bounded oracle sample."""
    name = ""
    dtype_name = "f64"
    unit = "GB/s"
    higher_is_better = True

    def config(self):
        return {}


class DenseWL(Workload):
    def __init__(self, n, dtype, arith="auto", strategy="fused", m=None):
        self.n, self.m = n, (m or n)
        self.dtype = dtype
        self.arith = arith
        self.strategy = strategy
        self.es = 8 if dtype == "f64" else 4
        self.dtype_name = dtype

    def setup(self, dev):
        import torch
        from paper_2507_13204_gb300 import api, workloads as W
        A, x = W.quadform_inputs(self.n, m=self.m, seed=0)
        td = torch.float64 if self.dtype == "f64" else torch.float32
        self.At = torch.tensor(A, dtype=td, device=dev)
        self.xt = torch.tensor(x, dtype=td, device=dev)
        self.A_host = A if self.dtype == "f64" else A.astype("float32").astype("float64")
        self.x_host = x if self.dtype == "f64" else x.astype("float32").astype("float64")
        self.p = api.QuadForm(self.At, strategy=self.strategy, arith=self.arith)
        self.gx = torch.empty(self.n, dtype=td, device=dev)
        self.f = torch.empty((), dtype=td, device=dev)
        self.fe = torch.empty((), dtype=td, device=dev)
        self.x_pin = torch.tensor(x, dtype=td).pin_memory()
        self.g_pin = torch.empty(self.n, dtype=td).pin_memory()
        self.f_pin = torch.empty((), dtype=td).pin_memory()
        self.td = td

    def step(self):
        self.p.grad(self.xt, gx=self.gx, f=self.f)

    def eval_step(self):
        self.p.eval(self.xt, f=self.fe)

    def e2e_step(self):
        self.p.grad_host(self.x_pin, self.g_pin, self.f_pin)

    @property
    def grad_bytes(self):  # A once, x in, gradient out
        return self.es * (self.m * self.n + 2 * self.n)

    @property
    def eval_bytes(self):
        return self.es * (self.m * self.n + self.n)

    @property
    def units_per_step(self):
        return self.grad_bytes / 1e9  # GB

    def dominant(self):
        """(name, algorithmic bytes per launch, fp64 flops per launch)"""
        return (self.grad_bytes - self.es * self.n, 4.0 * self.m * self.n)

    def h2d_d2h(self):
        return self.es * self.n, self.es * (self.n + 1)

    def config(self):
        cfg = {"workload": f"dense ||Ax||^2, A {self.m}x{self.n} {self.dtype.upper()} "
                           f"({self.es * self.m * self.n / 1e6:.0f} MB), value+grad wrt x",
               "strategy": self.strategy, "arith": self.arith,
               "l2": "inputs larger than L2 (A > 129 MB)"}
        if getattr(self, "p", None) is not None and self.dtype == "f64" and \
                self.p.workspace_bytes >= 8 * self.m * self.n:
            cfg["A_layout"] = ("float pairs (hi, lo) prepared once by kg_create, 8 B per entry "
                               "as in FP64; eval and grad stream that copy")
        return cfg

    def oracle_sample(self, budget_s=10.0):
        from oracle import oracle as O
        A, x = self.A_host, self.x_host
        return cpu_baseline_runs(
            lambda: O.quadform_grad_omp(A, x), lambda: O.quadform_grad(A, x),
            self.es * (self.m * self.n + 2 * self.n), f"full {self.m}x{self.n} value+grad",
            budget_s)

    def native_record(self, timed, peaks, box):
        """The same value-and-gradient in native FP64 arithmetic (IEEE FP64
        instructions throughout) on the same A: its step, forward, ratio, main
        kernel and FP64-ALU fraction."""
        import torch
        from paper_2507_13204_gb300 import _lib as L, api
        pn = api.QuadForm(self.At, strategy=self.strategy, arith="native")
        gx = torch.empty_like(self.gx)
        f, fe = torch.empty_like(self.f), torch.empty_like(self.fe)
        grad = lambda: pn.grad(self.xt, gx=gx, f=f)
        ev = lambda: pn.eval(self.xt, f=fe)
        for _ in range(3):
            grad()
            ev()
        t = timed(grad, 2)
        k = max(10, min(2000, int(500.0 / max(t, 1e-3))))
        L.kg_profile_enable(True)
        ms = timed(grad, k)
        kms, kn, kname = L.kg_profile_read()
        L.kg_profile_enable(False)
        ms_e = timed(ev, k)
        pn.sync()
        pn.close()
        kus = kms / max(kn, 1) * 1e3
        tf = 4.0 * self.m * self.n / 1e12 / (kus * 1e-6)
        peak, src = fp64_peak(peaks, box)
        return {"arith": "native", "ms_per_step": round(ms, 5), "ms_eval": round(ms_e, 5),
                "grad_over_eval_ratio": round(ms / ms_e, 4), "kernel": kname,
                "kernel_us": round(kus, 2), "fp64_tflops": round(tf, 4), "fp64_peak": round(peak, 4),
                "fp64_frac": round(tf / peak, 4), "fp64_peak_source": src,
                "hbm_gbs": round(self.grad_bytes / 1e9 / (ms * 1e-3), 1),
                "flops_per_launch": 4 * self.m * self.n, "steps": k}


class SparseWL(Workload):
    """Sparse ||Ax||^2, A 2^20 x 2^20 in CSR with 8..24 stored entries per row."""

    def __init__(self, m, dtype, strategy="auto", arith="auto"):
        self.m = m
        self.dtype = dtype
        self.dtype_name = dtype
        self.es = 8 if dtype == "f64" else 4
        self.strategy = strategy
        self.arith = arith

    def setup(self, dev):
        import torch
        from paper_2507_13204_gb300 import api, workloads as W
        A, x = W.spquadform_inputs(self.m)
        td = torch.float64 if self.dtype == "f64" else torch.float32
        if self.dtype == "f32":
            A.val = A.val.astype("float32").astype("float64")
            x = x.astype("float32").astype("float64")
        self.A, self.x_host, self.n, self.nnz = A, x, A.n, A.nnz
        self.rp = torch.tensor(A.rowptr, device=dev)
        self.cl = torch.tensor(A.col, device=dev)
        self.vl = torch.tensor(A.val, dtype=td, device=dev)
        self.xt = torch.tensor(x, dtype=td, device=dev)
        self.p = api.SpQuadForm(self.rp, self.cl, self.vl, self.n, strategy=self.strategy,
                                arith=self.arith)
        self.gx = torch.empty(self.n, dtype=td, device=dev)
        self.f = torch.empty((), dtype=td, device=dev)
        self.fe = torch.empty((), dtype=td, device=dev)
        self.x_pin = torch.tensor(x, dtype=td).pin_memory()
        self.g_pin = torch.empty(self.n, dtype=td).pin_memory()
        self.f_pin = torch.empty((), dtype=td).pin_memory()

    def l2_record(self, ms_grad, kernel_ms, strategy, box):
        """The bound of random access: every stored entry costs a gather of x in the
        forward and, in the reverse, a reduction into x-bar (ATOMIC) or a gather of y
        (the CSC strategy).  Their least time at this run's measured rates, against the
        step and the dominant kernel."""
        wide = self.dtype == "f64"  # FP64: 8-byte values (float pairs or doubles)
        g = box["fp64_gather_gops" if wide else "fp32_gather_gops"] * 1e9
        r = box["fp64_red_gops" if wide else "fp32_red_gops"] * 1e9
        rev = r if strategy == "atomic" else g
        t_min_ms = (self.nnz / g + self.nnz / rev) * 1e3
        return {"accesses_per_step": 2 * self.nnz, "gather_gops": round(g / 1e9, 1),
                "reverse": "red" if strategy == "atomic" else "gather",
                "reverse_gops": round(rev / 1e9, 1), "least_ms": round(t_min_ms, 5),
                "frac_of_step": round(t_min_ms / ms_grad, 4),
                "frac_of_kernel": round(t_min_ms / kernel_ms, 4) if strategy == "atomic" else None}

    def step(self):
        self.p.grad(self.xt, gx=self.gx, f=self.f)

    def eval_step(self):
        self.p.eval(self.xt, f=self.fe)

    def e2e_step(self):
        self.p.grad_host(self.x_pin, self.g_pin, self.f_pin)

    @property
    def grad_bytes(self):  # the CSR matrix once, x in, gradient out
        return 4 * (self.m + 1) + (4 + self.es) * self.nnz + 2 * self.es * self.n

    def dominant(self):
        if self.p.config[0] == "transpose":  # the column gather: CSC once, y in, gradient out
            return (4 * (self.n + 1) + (4 + self.es) * self.nnz + self.es * (self.m + self.n), None)
        return (self.grad_bytes, None)

    def h2d_d2h(self):
        return self.es * self.n, self.es * (self.n + 1)

    def config(self):
        return {"workload": f"sparse ||Ax||^2, A {self.m}x{self.n} CSR, 8..24 entries per row at "
                            f"uniform random columns ({self.nnz} stored), {self.dtype.upper()}, "
                            f"value+grad wrt x",
                "strategy": self.strategy, "arith": self.arith,
                "l2": "inputs larger than L2 (CSR > 129 MB)"}

    def oracle_sample(self, budget_s=10.0):
        from oracle import oracle as O
        t0 = time.perf_counter()
        reps = 0
        while True:
            O.spquadform_grad(self.A.rowptr, self.A.col, self.A.val, self.x_host)
            reps += 1
            if time.perf_counter() - t0 >= budget_s or reps >= 20:
                break
        dt = time.perf_counter() - t0
        return reps * self.grad_bytes / 1e9 / dt, f"{reps} x full value+grad (oracle, 1 thread)"


class TetWL(Workload):
    def __init__(self, a, dtype, strategy="auto", arith="auto"):
        self.a = a
        self.dtype = dtype
        self.dtype_name = dtype
        self.es = 8 if dtype == "f64" else 4
        self.strategy = strategy
        self.arith = arith

    def setup(self, dev):
        import torch
        from paper_2507_13204_gb300 import api, workloads as W
        mesh, u = W.tet_inputs(self.a)
        td = torch.float64 if self.dtype == "f64" else torch.float32
        self.mesh, self.u_host = mesh, u
        self.ne, self.nv = mesh.ne, mesh.nv
        self.conn = torch.tensor(mesh.conn, device=dev)
        self.G = torch.tensor(mesh.G, dtype=td, device=dev)
        self.u = torch.tensor(u, dtype=td, device=dev)
        self.p = api.TetEnergy(self.conn, self.G, mesh.nv, strategy=self.strategy,
                               mode="recompute", arith=self.arith)
        self.gu = torch.empty(mesh.nv, dtype=td, device=dev)
        self.f = torch.empty((), dtype=td, device=dev)
        self.fe = torch.empty((), dtype=td, device=dev)
        self.x_pin = torch.tensor(u, dtype=td).pin_memory()
        self.g_pin = torch.empty(mesh.nv, dtype=td).pin_memory()
        self.f_pin = torch.empty((), dtype=td).pin_memory()

    def step(self):
        self.p.grad(self.u, gx=self.gu, f=self.f)

    def eval_step(self):
        self.p.eval(self.u, f=self.fe)

    def e2e_step(self):
        self.p.grad_host(self.x_pin, self.g_pin, self.f_pin)

    @property
    def eval_bytes(self):  # conn + G streamed, u read once
        return self.ne * (16 + 12 * self.es) + self.nv * self.es

    @property
    def grad_bytes(self):  # + gradient written once
        return self.eval_bytes + self.nv * self.es

    @property
    def units_per_step(self):
        return self.grad_bytes / 1e9

    def dominant(self):
        return (self.grad_bytes, None)

    def h2d_d2h(self):
        return self.es * self.nv, self.es * (self.nv + 1)

    def config(self):
        return {"workload": f"tet-mesh energy sum_e log1p(|G_e u_e|^2), {self.a}^3 cubes x 6 tets "
                            f"({self.ne} tets, {self.nv} vertices, random relabelling), "
                            f"{self.dtype.upper()}, value+grad wrt u",
                "strategy": self.strategy, "arith": self.arith,
                "l2": "inputs larger than L2 (conn+G > 129 MB)"}

    def oracle_sample(self, budget_s=10.0):
        from oracle import oracle as O
        conn, G, u = self.mesh.conn, self.mesh.G, self.u_host
        ne1 = min(self.ne, 1_000_000)
        c1, G1 = conn[:ne1], G[:ne1]
        return cpu_baseline_runs(
            lambda: O.tet_grad_omp(conn, G, u), lambda: O.tet_grad(c1, G1, u),
            self.ne * (16 + 12 * self.es) + 2 * self.nv * self.es,
            f"full {self.ne}-tet value+grad", budget_s,
            serial_bytes=ne1 * (16 + 12 * self.es) + 2 * self.nv * self.es,
            serial_what=f"value+grad of the first {ne1} tets")


class HvpWL(TetWL):
    """Hessian-vector product of the tet energy (forward mode over the reverse pass) on the
    100^3 x 6 mesh; the comparison line (ms_eval, ratio) is the value+grad of the same mesh."""

    def setup(self, dev):
        import torch
        super().setup(dev)
        td = self.u.dtype
        v = np.random.default_rng(43).uniform(-1.0, 1.0, self.nv)
        self.v = torch.tensor(v, dtype=td, device=dev)
        self.hv = torch.empty(self.nv, dtype=td, device=dev)
        self.v_pin = torch.tensor(v, dtype=td).pin_memory()
        self.stream = torch.cuda.current_stream()

    def step(self):
        self.p.hvp(self.u, self.v, hv=self.hv)

    def eval_step(self):  # the comparison: value+grad
        self.p.grad(self.u, gx=self.gu, f=self.f)

    def e2e_step(self):
        self.u.copy_(self.x_pin, non_blocking=True)
        self.v.copy_(self.v_pin, non_blocking=True)
        self.p.hvp(self.u, self.v, hv=self.hv)
        self.g_pin.copy_(self.hv, non_blocking=True)
        self.stream.synchronize()

    @property
    def grad_bytes(self):  # conn + G streamed, u and v read, hv written
        return self.ne * (16 + 12 * self.es) + 3 * self.nv * self.es

    def h2d_d2h(self):
        return 2 * self.es * self.nv, self.es * self.nv

    def config(self):
        c = super().config()
        c["workload"] = c["workload"].replace("value+grad wrt u", "Hessian-vector product H(u) v")
        c["comparison"] = "ms_eval / grad_over_eval_ratio here are the value+grad of the same mesh"
        return c

    def oracle_sample(self, budget_s=10.0):
        from oracle import oracle as O
        ne = min(self.ne, 1_000_000)
        conn, G = self.mesh.conn[:ne], self.mesh.G[:ne]
        v = np.random.default_rng(43).uniform(-1.0, 1.0, self.nv)
        t0 = time.perf_counter()
        reps = 0
        while True:
            O.tet_hvp(conn, G, self.u_host, v)
            reps += 1
            if time.perf_counter() - t0 >= budget_s or reps >= 20:
                break
        dt = time.perf_counter() - t0
        b = reps * (ne * (16 + 12 * self.es) + 3 * self.nv * self.es)
        return b / 1e9 / dt, f"{reps} x Hessian-vector product on the first {ne} tets (oracle, 1 thread)"


class LaplaceWL(Workload):
    """The paper's E1 example at n = 10000 (data 80 KB: launch-bound, like the paper)."""

    def __init__(self, n, strategy="fused"):
        self.n = n
        self.es = 8
        self.strategy = strategy
        self.unit = "grads/s"

    def setup(self, dev):
        import torch
        from paper_2507_13204_gb300 import api, workloads as W
        x, b = W.laplace1d_inputs(self.n)
        self.x_host, self.b_host = x, b
        self.b = torch.tensor(b, device=dev)
        self.x = torch.tensor(x, device=dev)
        self.p = api.Laplace1D(self.b, strategy=self.strategy)
        self.gx = torch.empty(self.n, dtype=torch.float64, device=dev)
        self.gb = torch.empty(self.n, dtype=torch.float64, device=dev)
        self.f = torch.empty((), dtype=torch.float64, device=dev)
        self.fe = torch.empty((), dtype=torch.float64, device=dev)
        self.x_pin = torch.tensor(x).pin_memory()
        self.g_pin = torch.empty(self.n, dtype=torch.float64).pin_memory()
        self.f_pin = torch.empty((), dtype=torch.float64).pin_memory()

    def step(self):
        self.p.grad(self.x, gx=self.gx, f=self.f, gdata=self.gb)

    def eval_step(self):
        self.p.eval(self.x, f=self.fe)

    def e2e_step(self):
        self.p.grad_host(self.x_pin, self.g_pin, self.f_pin)

    grad_bytes = property(lambda self: 8 * 4 * self.n)
    eval_bytes = property(lambda self: 8 * 2 * self.n)
    units_per_step = 1.0

    def dominant(self):
        return (self.grad_bytes, None)

    def h2d_d2h(self):
        return 8 * self.n, 8 * (self.n + 1)

    def config(self):
        return {"workload": f"paper example ||A(3x)-b||^2, 1-D Laplacian, n={self.n} FP64",
                "strategy": self.strategy, "l2": "resident in L2 (160 KB)"}

    def oracle_sample(self, budget_s=10.0):
        from oracle import oracle as O
        t0 = time.perf_counter()
        reps = 0
        while time.perf_counter() - t0 < budget_s and reps < 200000:
            O.laplace1d_grad(self.x_host, self.b_host)
            reps += 1
        return reps / (time.perf_counter() - t0), f"{reps} x value+grad at n={self.n} (oracle, 1 thread)"


class BatchedWL(Workload):
    """4096 dense ||A_k x_k||^2 (n_k log-uniform in [32, 2048]) + 512 tet meshes
    (1e3..1e5 tets), FP64, all gradients in one persistent launch (CUDA graph);
    compared with the per-instance launch loop."""
    unit = "grads/s"

    def __init__(self, ndense=4096, ntet=512, arith="auto", strategy="auto", nrange=None, limit=0):
        """nrange (lo, hi), limit: only the first `limit` dense instances with lo <= n < hi of
        the batch's draw, no tets (a profiling case of the same instances)."""
        self.ndense, self.ntet, self.arith, self.strategy = ndense, ntet, arith, strategy
        self.nrange, self.limit = nrange, limit
        self.ndraw, self.ntet_draw = ndense, ntet  # sizes of the draws (setup() counts the picks)
        self.es = 8

    def instances(self):
        """(indices k of the dense draw, their n_k, the tet boxes) of this batch."""
        from paper_2507_13204_gb300 import workloads as W
        drawn = W.batched_dense_sizes(self.ndraw)
        ks = [k for k, n in enumerate(drawn)
              if self.nrange is None or self.nrange[0] <= n < self.nrange[1]]
        if self.limit:
            ks = ks[:self.limit]
        return ks, [int(drawn[k]) for k in ks], (W.batched_tet_boxes(self.ntet_draw) if self.ntet_draw else [])

    def setup(self, dev):
        import torch
        from paper_2507_13204_gb300 import api, workloads as W
        ks, sizes, boxes = self.instances()
        self.sizes, self.boxes = sizes, boxes
        self.ndense, self.ntet = len(sizes), len(boxes)
        probs, self.A, nx = [], [], []
        self.tets = []
        for k, n in zip(ks, sizes):
            A, x = W.batched_dense_device(k, int(n), dev)
            self.A.append((A, x))
            probs.append(api.QuadForm(A, arith=self.arith))
            nx.append(int(n))
        for k, box in enumerate(boxes):
            mesh, u = W.batched_tet_instance(k, box)
            conn = torch.tensor(mesh.conn, device=dev)
            G = torch.tensor(mesh.G, device=dev)
            self.tets.append((mesh, u, conn, G))
            probs.append(api.TetEnergy(conn, G, mesh.nv, arith=self.arith))
            nx.append(mesh.nv)
        self.probs = probs
        offs = [0]
        for v in nx:
            offs.append(offs[-1] + ((v + 1) // 2) * 2)  # 16-byte aligned views
        self.xbuf = torch.zeros(offs[-1], dtype=torch.float64, device=dev)
        self.gbuf = torch.zeros(offs[-1], dtype=torch.float64, device=dev)
        self.fbuf = torch.zeros(len(nx), dtype=torch.float64, device=dev)
        self.xs = [self.xbuf[offs[i]:offs[i] + nx[i]] for i in range(len(nx))]
        self.gxs = [self.gbuf[offs[i]:offs[i] + nx[i]] for i in range(len(nx))]
        self.fs = [self.fbuf[i] for i in range(len(nx))]
        for i, (A, x) in enumerate(self.A):
            self.xs[i].copy_(x)
        for j, (mesh, u, _, _) in enumerate(self.tets):
            self.xs[self.ndense + j].copy_(torch.tensor(u, device=dev))
        # float-pair copies of every dense A without one (the n < 1024 instances, 4.2 GB)
        self.batch = api.Batch(probs, arith=self.arith, strategy=self.strategy, budget_bytes=8 << 30)
        self.bound = self.batch.bind(self.xs, self.fs, self.gxs)  # pointer tables built once
        self.x_pin = self.xbuf.cpu().pin_memory()
        self.g_pin = torch.empty_like(self.gbuf, device="cpu").pin_memory()
        self.f_pin = torch.empty_like(self.fbuf, device="cpu").pin_memory()
        self.count = len(nx)
        self.dtype_name = "f64"
        dense_b = sum(8 * (int(n) * int(n) + 2 * int(n)) for n in sizes)
        tet_b = sum(t[0].ne * (16 + 96) + 2 * t[0].nv * 8 for t in self.tets)
        self.grad_bytes = dense_b + tet_b
        self.eval_bytes = self.grad_bytes

    def step(self):
        self.batch.grad(self.bound)

    def eval_step(self):  # the per-instance launch loop (the comparison)
        self.batch.grad_loop(self.bound)

    def e2e_step(self):
        import torch
        self.xbuf.copy_(self.x_pin, non_blocking=True)
        self.batch.grad(self.bound)
        self.g_pin.copy_(self.gbuf, non_blocking=True)
        self.f_pin.copy_(self.fbuf, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    @property
    def units_per_step(self):
        return self.count

    def dominant(self):
        return (self.grad_bytes, None)

    def h2d_d2h(self):
        return self.xbuf.numel() * 8, self.gbuf.numel() * 8 + self.fbuf.numel() * 8

    @property
    def p(self):
        return self.probs[0]

    def config(self):
        pick = ("" if self.nrange is None else
                f", the first with {self.nrange[0]} <= n_k < {self.nrange[1]} of the 4096 drawn")
        return {"workload": f"batched: {self.ndense} dense ||A_k x_k||^2 (n_k log-uniform "
                            f"[32, 2048]{pick}) + {self.ntet} tet meshes (1e3..1e5 tets), FP64, all "
                            f"value+grads in one persistent launch (CUDA graph); float-pair "
                            f"copies of the data made at create",
                "l2": f"inputs larger than L2 ({self.grad_bytes / 1e9:.1f} GB)",
                "comparison": "ms_eval / grad_over_eval_ratio here are the per-instance launch loop"}

    def oracle_sample(self, budget_s=10.0):
        from oracle import oracle as O
        t0 = time.perf_counter()
        done = 0
        k = 0
        host = []
        for A, x in self.A[:64]:
            host.append(("d", A.cpu().numpy(), x.cpu().numpy()))
        for mesh, u, _, _ in self.tets[:8]:
            host.append(("t", mesh, u))
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < budget_s and k < 4 * len(host):
            h = host[k % len(host)]
            if h[0] == "d":
                O.quadform_grad(h[1], h[2])
            else:
                O.tet_grad(h[1].conn, h[1].G, h[2])
            done += 1
            k += 1
        dt = time.perf_counter() - t0
        nd, nt = min(64, len(self.A)), min(8, len(self.tets))
        return done / dt, (f"{done} instances (first {nd} dense + first {nt} tet instances, cycled; "
                           f"oracle, 1 thread)")


class AutogradWL(Workload):
    """Gradient descent u <- u - 0.01 grad f(u) through torch.autograd
    (KGTetEnergy) on the 6e6-tet mesh; step = one forward + backward + update.
    The main policy is the tape (forward records c_e, backward scatters it);
    recompute (backward reruns the fused value-and-gradient kernel) is timed
    beside it as the comparison."""
    unit = "steps/s"
    ETA = 0.01

    def __init__(self, a=100, dtype="f64", arith="auto"):
        self.a, self.dtype, self.arith = a, dtype, arith
        self.dtype_name = dtype
        self.es = 8 if dtype == "f64" else 4

    def setup(self, dev):
        import torch
        from paper_2507_13204_gb300 import api, autograd, workloads as W
        mesh, u = W.tet_inputs(self.a)
        td = torch.float64 if self.dtype == "f64" else torch.float32
        self.mesh, self.u_host = mesh, u
        self.ne, self.nv = mesh.ne, mesh.nv
        conn = torch.tensor(mesh.conn, device=dev)
        G = torch.tensor(mesh.G, dtype=td, device=dev)
        self.p_tape = api.TetEnergy(conn, G, mesh.nv, mode="tape", arith=self.arith)
        self.p_rec = api.TetEnergy(conn, G, mesh.nv, mode="recompute", arith=self.arith)
        self.ag = autograd
        self.u = torch.tensor(u, dtype=td, device=dev)
        self.u_rec = self.u.clone()
        self.x_pin = torch.tensor(u, dtype=td).pin_memory()
        self.g_pin = torch.empty(mesh.nv, dtype=td).pin_memory()
        self.f_pin = torch.empty((), dtype=td).pin_memory()
        self.p = self.p_tape
        self.tape_bytes = 4 * self.ne * self.es

    def _step(self, prob, u, policy):
        import torch
        ut = u.requires_grad_(True)
        f = self.ag.KGTetEnergy.apply(ut, prob, policy)
        (g,) = torch.autograd.grad(f, ut)
        return (ut.detach() - self.ETA * g).detach()

    def step(self):
        self.u = self._step(self.p_tape, self.u, "tape")

    def eval_step(self):  # the recompute policy (the comparison)
        self.u_rec = self._step(self.p_rec, self.u_rec, "recompute")

    def e2e_step(self):
        self.p_tape.grad_host(self.x_pin, self.g_pin, self.f_pin)

    @property
    def grad_bytes(self):  # tape: forward streams conn+G and writes the tape; backward reads conn+tape
        return self.ne * (16 + 12 * self.es) + 4 * self.ne * self.es + self.ne * 16 + \
            4 * self.ne * self.es + 3 * self.nv * self.es

    def dominant(self):
        return (self.ne * (16 + 12 * self.es) + 4 * self.ne * self.es + self.nv * self.es, None)

    def h2d_d2h(self):
        return self.es * self.nv, self.es * (self.nv + 1)

    def config(self):
        return {"workload": f"torch.autograd.Function KGTetEnergy, gradient descent (eta 0.01) on "
                            f"the {self.a}^3 x 6 = {self.ne}-tet mesh, {self.dtype.upper()}",
                "policy": "tape (main) vs recompute (ms_eval, grad_over_eval_ratio)",
                "tape_bytes": self.tape_bytes,
                "l2": "inputs larger than L2"}

    def oracle_sample(self, budget_s=10.0):
        from oracle import oracle as O
        ne = min(self.ne, 500_000)
        conn, G = self.mesh.conn[:ne], self.mesh.G[:ne]
        t0 = time.perf_counter()
        steps = 0
        u = self.u_host.copy()
        while time.perf_counter() - t0 < budget_s and steps < 50:
            u, _ = O.tet_descent(conn, G, u, self.ETA, 1)
            steps += 1
        dt = time.perf_counter() - t0
        return steps * ne / self.ne / dt, (f"{steps} descent steps on the first {ne} tets, "
                                           f"scaled to the full mesh (oracle, 1 thread)")


def make_workload(name: str, arith: str, size: int = 0, rows: int = 0, strategy: str = ""):
    if name == "autograd":
        return AutogradWL(size or 100, "f64", arith=arith)
    if name == "autograd32":
        return AutogradWL(size or 100, "f32")
    if name == "batched":
        return BatchedWL(size or 4096, max(1, (size or 4096) // 8), arith=arith,
                         strategy=strategy or "auto")
    if name == "batched_big":  # profiling case: the batch's first dense instances of 1024 <= n < 2048
        return BatchedWL(4096, 0, arith=arith, strategy=strategy or "auto", nrange=(1024, 2048),
                         limit=size or 96)
    if name == "dense":
        return DenseWL(size or 10000, "f64", arith=arith, m=rows or None)
    if name == "dense32":
        return DenseWL(size or 10000, "f32", m=rows or None)
    if name == "dense64":
        return DenseWL(64, "f64", arith=arith)
    if name == "tet":
        return TetWL(size or 100, "f64", strategy=strategy or "auto", arith=arith)
    if name == "tet32":
        return TetWL(size or 100, "f32", strategy=strategy or "auto")
    if name == "tetcsr":
        return TetWL(size or 100, "f64", strategy="csr", arith=arith)
    if name == "hvp":
        return HvpWL(size or 100, "f64", strategy=strategy or "auto", arith=arith)
    if name == "hvp32":
        return HvpWL(size or 100, "f32", strategy=strategy or "auto")
    if name == "sparse":
        return SparseWL(size or (1 << 20), "f64", strategy=strategy or "auto", arith=arith)
    if name == "sparse32":
        return SparseWL(size or (1 << 20), "f32", strategy=strategy or "auto")
    if name == "laplace":
        return LaplaceWL(size or 10000)
    if name == "laplace_atomic":
        return LaplaceWL(size or 10000, strategy="atomic")
    raise SystemExit(f"unknown workload {name}")


# ------------------------------------------------------------------ traffic
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one steady-state launch of the
# dominant kernel at the default workload sizes, from one full-size ncu capture each (one
# pass; see profiles/).  A value is reported only while the kernel's sources hash to the
# fingerprint it was taken with; after any change to them the field is null until re-measured.
_CSRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2507_13204_gb300", "csrc")
_TRAFFIC = {
    ('dense', 'f64'): (816462080, ['quadform_pair.cu', 'kg_pair.cuh', 'kg_device.cuh'],
                       '78d8ecfe03606423'),
    ('dense32', 'f32'): (405942784, ['quadform_f32.cu', 'kg_pair.cuh', 'kg_device.cuh'],
                         '801a828817b83d19'),
    ('tet', 'f64'): (711157760, ['tet_pair.cu', 'kg_tet_elem.cuh', 'kg_pair.cuh', 'kg_device.cuh'],
                     '33085ea1051816f5'),
    ('tet32', 'f32'): (469459712, ['tet_tile.cu', 'kg_tet_elem.cuh', 'kg_pair.cuh', 'kg_device.cuh'],
                       '166f724fdbe0f6dd'),
    ('tetcsr', 'f64'): (787957760, ['tet_tile.cu', 'kg_tet_elem.cuh', 'kg_pair.cuh', 'kg_device.cuh'],
                        '166f724fdbe0f6dd'),
    ('batched', 'f64'): (18503473152, ['batched.cu', 'kg_tet_elem.cuh', 'kg_pair.cuh', 'kg_device.cuh'],
                         '2bc7e7b9c7b540ad'),
}


def _code_only(text: str) -> str:
    """C/CUDA source without its comments and with whitespace runs collapsed, so that
    editing a comment keeps a kernel's fingerprint (no string in these sources holds
    a comment marker)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def source_fingerprint(files) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in files:
        h.update(f.encode())
        with open(os.path.join(_CSRC, f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str, dtype: str, default_sizes: bool):
    """DRAM bytes per launch of the dominant kernel, or None (other sizes, no capture, or
    the kernel's sources changed since the capture)."""
    rec = _TRAFFIC.get((workload, dtype))
    if rec is None or not default_sizes:
        return None
    nbytes, files, fp = rec
    try:
        return nbytes if source_fingerprint(files) == fp else None
    except OSError:
        return None


# ------------------------------------------------------------------ ranks
def sync_max(values, dist=None, device="cpu"):
    """Max over ranks of each entry of `values` (identity without a process group)."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Units of all ranks per second, timed by the slowest rank (weak scaling: every
    rank runs its own replica of the workload)."""
    return world * units_per_rank / (ms_max * 1e-3)


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="timed steps (0: about 3 s worth)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="kg", choices=["kg", "reference"])
    ap.add_argument("--workload", default="dense")
    ap.add_argument("--arith", default="auto", choices=["auto", "native", "pair"])
    ap.add_argument("--size", type=int, default=0,
                    help="problem size override (dense n, tet cubes per axis, 1-D n) for small "
                         "profiling cases; the default is the full workload")
    ap.add_argument("--rows", type=int, default=0, help="dense: rows of A (default: square)")
    ap.add_argument("--strategy", default="", choices=["", "atomic", "shared", "warp", "tile", "csr",
                                                       "transpose"],
                    help="tet, batched, sparse: reverse-pass scatter strategy (default: the "
                         "library's choice)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "laplace_sweep":
        return run_laplace_sweep(args)

    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    from paper_2507_13204_gb300 import _lib as L, build as B
    if rank == 0 or world == 1:
        B.build()
    if dist:
        dist.barrier()
    wl = make_workload(args.workload, args.arith, args.size, args.rows, args.strategy)
    wl.setup(dev)
    stream = torch.cuda.current_stream()
    peaks = load_peaks()

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    def timed(fn, k):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1) / k  # ms per step

    for _ in range(args.warmup):
        wl.step()
        wl.eval_step()
    torch.cuda.synchronize()
    try:  # FP64 / FP32 FMA and red rates of this GPU (a few ms)
        box = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in L.kg_measure_box().items()}
    except Exception as e:  # noqa: BLE001
        box = {"error": str(e)}
    wl.step()
    launches_per_step = L.kg_last_launch_count()
    wl.eval_step()
    launches_eval = L.kg_last_launch_count()
    # step count: exactly --steps, else about 3 s of gradient steps
    t_probe = timed(wl.step, 3)
    K = args.steps if args.steps > 0 else max(10, min(20000, int(3000.0 / max(t_probe, 1e-3))))

    def busy(fn, seconds):
        """Untimed steps for `seconds` of wall time, synchronising every few
        steps so that the host never runs far ahead of the GPU."""
        chunk = max(1, int(20.0 / max(t_probe, 1e-3)))  # about 20 ms of steps
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < seconds:
            for _ in range(chunk):
                fn()
            torch.cuda.synchronize()

    # Clock record: nvidia-smi samples every 200 ms from before a second of
    # untimed steps, through the timed steps, to half a second of untimed steps
    # after them, so that it holds samples of this workload under load however
    # short the timed region is.
    clocks = ClockSampler(local)
    clocks.start()
    clocks.wait_first_row()
    busy(wl.step, 1.0)
    L.kg_profile_enable(True)
    ms_grad = timed(wl.step, K)
    kern_ms, kern_n, kern_name = L.kg_profile_read()
    L.kg_profile_enable(False)
    busy(wl.step, 0.5)
    clk = clocks.stop()
    if clk is not None:
        clk["window"] = ("nvidia-smi every 200 ms over 1 s of untimed steps, the timed steps "
                         "and 0.5 s of untimed steps of the same workload")
    t_probe_e = timed(wl.eval_step, 1)
    Ke = max(3, min(K, int(3000.0 / max(t_probe_e, 1e-3))))
    ms_eval = timed(wl.eval_step, Ke)

    ms_grad, ms_eval = sync_max([ms_grad, ms_eval], dist, dev)

    # end-to-end: host buffers through the C ABI, copies inside the timed region
    K2 = max(5, min(K, int(2000.0 / max(ms_grad, 1e-3))))
    for _ in range(2):
        wl.e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(K2):
        wl.e2e_step()
    barrier()
    ms_e2e = (time.perf_counter() - t0) * 1e3 / K2
    (ms_e2e,) = sync_max([ms_e2e], dist, dev)

    native = None
    if isinstance(wl, DenseWL) and wl.dtype == "f64" and wl.p.config[2] == "pair":
        native = wl.native_record(timed, peaks, box)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    if isinstance(wl, (LaplaceWL, AutogradWL)):
        units = 1.0
    elif isinstance(wl, BatchedWL):
        units = wl.count
    else:
        units = wl.grad_bytes / 1e9
    value = whole_job_rate(units, world, ms_grad)
    e2e_value = whole_job_rate(units, world, ms_e2e)
    # dominant kernel roofline
    per_launch_ms = kern_ms / max(kern_n, 1)
    dbytes, dflops = wl.dominant()
    ach_gbs = dbytes / 1e9 / (per_launch_ms * 1e-3) if per_launch_ms > 0 else 0.0
    default_sizes = args.size == 0 and args.rows == 0 and args.strategy == "" and args.arith == "auto"
    traffic = recorded_traffic(args.workload, wl.dtype_name, default_sizes)
    roof = {"bound": "hbm", "achieved": round(ach_gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(ach_gbs / peaks["hbm_gbs"], 4), "traffic": traffic,
            "kernel": kern_name, "kernel_us": round(per_launch_ms * 1e3, 2),
            "peak_source": f"{peaks["hbm_src"]} copy bandwidth"}
    strategy, mode, arith = wl.p.config
    if isinstance(wl, BatchedWL):
        arith, nitems, bgrid = wl.batch.config
        strategy, mode = f"batched ({nitems} work items, {bgrid} CTAs)", "recompute"
    native64 = wl.dtype_name == "f64" and arith == "native"
    if dflops and native64 and per_launch_ms > 0:
        ach_tf = dflops / 1e12 / (per_launch_ms * 1e-3)
        fpk, fsrc = fp64_peak(peaks, box)
        frac_alu = ach_tf / fpk
        if frac_alu > roof["frac"]:
            roof = {"bound": "alu", "achieved": round(ach_tf, 4), "peak": round(fpk, 4),
                    "unit": "TFLOP/s", "frac": round(frac_alu, 4), "traffic": None,
                    "kernel": kern_name, "kernel_us": round(per_launch_ms * 1e3, 2),
                    "peak_source": fsrc,
                    "hbm_gbs": round(ach_gbs, 1), "hbm_frac": round(ach_gbs / peaks["hbm_gbs"], 4)}

    out = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": wl.unit,
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": round(ms_grad, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": wl.dtype_name,
        "data": "synthetic (seeded numpy PCG64 draws)",
        "config": {**wl.config(), "strategy": strategy, "mode": mode, "arith": arith},
        "grad_over_eval_ratio": round(ms_grad / ms_eval, 4),
        "ms_eval": round(ms_eval, 5),
        **({"autograd": {"tape_ms_per_step": round(ms_grad, 4), "recompute_ms_per_step": round(ms_eval, 4),
                         "tape_bytes": wl.tape_bytes, "tape_vs_recompute_speedup": round(ms_eval / ms_grad, 3)}}
           if isinstance(wl, AutogradWL) else {}),
        "pct_of_hbm_peak": round(100 * value / world / peaks["hbm_gbs"], 2) if wl.unit == "GB/s" else None,
        "pct_of_8tbs_nominal": round(100 * value / world / 8000.0, 2) if wl.unit == "GB/s" else None,
        "roofline": roof,
        "e2e": {"value": round(e2e_value, 3), "unit": wl.unit,
                "h2d_bytes_per_step": wl.h2d_d2h()[0], "d2h_bytes_per_step": wl.h2d_d2h()[1],
                "ms_per_step": round(ms_e2e, 5), "api": "kg_grad_host (pinned host buffers)"},
        "gpu_launches": launches_per_step * K,
        **({"batched": {"loop_grads_per_s": round(wl.count * 1000.0 / ms_eval, 1),
                        "speedup_vs_loop": round(ms_eval / ms_grad, 2),
                        "aggregate_gbs": round(wl.grad_bytes / 1e9 / (ms_grad * 1e-3), 1),
                        "instances": wl.count}} if isinstance(wl, BatchedWL) else {}),
        "launches_per_step": {"grad": launches_per_step, "eval": launches_eval},
        "clocks": clk,
        **({"native_f64": native} if native else {}),
        **({"l2_random": wl.l2_record(ms_grad, per_launch_ms, strategy, box)}
           if isinstance(wl, SparseWL) and "error" not in box else {}),
        "box": box,
    }
    if world == 1 and not args.no_cpu_baseline:
        res = wl.oracle_sample()
        if isinstance(res, dict):
            out["cpu_baseline"] = {"value": res["value"], "unit": wl.unit, "cores": res["cores"],
                                   "kind": "oracle", "sample": res["sample"],
                                   **{k: v for k, v in res.items()
                                      if k not in ("value", "cores", "kind", "sample")}}
        else:
            v, sample = res
            out["cpu_baseline"] = {"value": round(v, 4), "unit": wl.unit, "cores": 1, "kind": "oracle",
                                   "sample": sample}
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def run_laplace_sweep(args):
    """The paper's experiment (Sec. 4): f and its gradient for n = 1, 100, ..., 10000,
    timed per call.  Two clocks: host wall-clock per call including a stream
    synchronisation (the paper's f returns a host scalar), and device time
    (CUDA events over back-to-back calls).  Ratio = t(grad) / t(f)."""
    import statistics as st
    import torch
    from paper_2507_13204_gb300 import _lib as L, api, build as B, workloads as W
    B.build()
    dev = torch.device("cuda", 0)
    ns = [1] + list(range(100, 10001, 100))
    reps = max(20, args.steps or 50)
    out = {}
    for strategy in ("fused", "atomic"):
        rows = []
        for n in ns:
            x, b = W.laplace1d_inputs(n)
            bt = torch.tensor(b, device=dev)
            xt = torch.tensor(x, device=dev)
            p = api.Laplace1D(bt, strategy=strategy)
            f = torch.empty((), dtype=torch.float64, device=dev)
            gx = torch.empty(n, dtype=torch.float64, device=dev)
            gb = torch.empty(n, dtype=torch.float64, device=dev)
            ev = lambda: p.eval(xt, f=f)
            gr = lambda: p.grad(xt, gx=gx, f=f, gdata=gb)
            res = {}
            for name, fn in (("f", ev), ("grad", gr)):
                for _ in range(5):
                    fn()
                torch.cuda.synchronize()
                wall = []
                for _ in range(reps):
                    t0 = time.perf_counter()
                    fn()
                    torch.cuda.current_stream().synchronize()
                    wall.append(time.perf_counter() - t0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    fn()
                e1.record()
                torch.cuda.synchronize()
                res[name] = (st.median(wall) * 1e6, e0.elapsed_time(e1) * 1e3 / reps)
                launches = L.kg_last_launch_count()
                res[name + "_launches"] = launches
            rows.append((n, res))
            p.close()
        wr = [r["grad"][0] / r["f"][0] for _, r in rows]
        dr = [r["grad"][1] / r["f"][1] for _, r in rows]
        out[strategy] = {
            "wall_ratio_max": round(max(wr), 3), "wall_ratio_mean": round(sum(wr) / len(wr), 3),
            "device_ratio_max": round(max(dr), 3), "device_ratio_mean": round(sum(dr) / len(dr), 3),
            "wall_us_f_n1": round(rows[0][1]["f"][0], 2), "wall_us_grad_n1": round(rows[0][1]["grad"][0], 2),
            "wall_us_f_n10000": round(rows[-1][1]["f"][0], 2),
            "wall_us_grad_n10000": round(rows[-1][1]["grad"][0], 2),
            "device_us_f_n10000": round(rows[-1][1]["f"][1], 3),
            "device_us_grad_n10000": round(rows[-1][1]["grad"][1], 3),
            "launches": {"f": rows[-1][1]["f_launches"], "grad": rows[-1][1]["grad_launches"]},
        }
    line = {"metric": "gradient/function wall-clock ratio (paper's 1-D Laplacian example, n = 1..10000)",
            "value": out["fused"]["wall_ratio_max"], "unit": "ratio", "n_gpus": 1, "steps": reps,
            "warmup": 5, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": round(out["fused"]["wall_ratio_max"] / 2.17, 3), "dtype": "f64",
            "data": "synthetic (seeded numpy PCG64 draws)",
            "config": {"workload": "paper example f(x,b) = ||A(3x) - b||^2, A = tridiag(-1,2,-1), "
                                   "n = 1, 100, ..., 10000 (101 sizes)",
                       "baseline": "paper's max ratio 2.17 (MI250X), 1.81 (H100), 1.99 (PVC)"},
            "fused": out["fused"], "paper_six_kernel_atomic": out["atomic"]}
    print(json.dumps(line), flush=True)


def run_reference(args, rank, world):
    """The CPU oracle as the reference arm: rank 0 only, bounded samples."""
    if rank != 0:
        return
    wl = make_workload(args.workload, "auto", args.size, args.rows)
    # inputs only (no GPU): build the host arrays the oracle needs
    from paper_2507_13204_gb300 import workloads as W
    from oracle import oracle as O
    O.build()
    cores = 1
    if isinstance(wl, DenseWL):
        A, x = W.quadform_inputs(wl.n, m=wl.m, seed=0)
        if wl.dtype == "f32":
            A, x = A.astype("float32").astype("float64"), x.astype("float32").astype("float64")
        unit_bytes = wl.es * (wl.m * wl.n + 2 * wl.n)
        try:
            cores = O.omp_threads()
            fn = lambda: O.quadform_grad_omp(A, x)
            sample = (f"full value+grad of the {wl.m}x{wl.n} problem per step (oracle, OpenMP "
                      f"build, {cores} threads)")
        except Exception:  # noqa: BLE001  (no OpenMP build: serial oracle on 1000 rows)
            rows = min(1000, A.shape[0])
            A = A[:rows].copy()
            unit_bytes = wl.es * (rows * wl.n + 2 * wl.n)
            fn = lambda: O.quadform_grad(A, x)
            sample = f"value+grad of the first {rows} rows of the {wl.m}x{wl.n} problem per step"
        to_value = lambda s: unit_bytes / 1e9 / s
    elif isinstance(wl, AutogradWL):
        mesh, u = W.tet_inputs(wl.a)
        wl.mesh, wl.u_host, wl.ne, wl.nv = mesh, u, mesh.ne, mesh.nv
        wl.tape_bytes = 4 * wl.ne * wl.es
        ne = min(mesh.ne, 500_000)
        conn, G = mesh.conn[:ne], mesh.G[:ne]
        state = {"u": u.copy()}

        def fn():
            _, g = O.tet_grad(conn, G, state["u"])
            state["u"] = state["u"] - wl.ETA * g

        sample = (f"one descent step (oracle gradient and update) on the first {ne} tets of the "
                  f"{wl.a}^3 mesh per step, scaled to the full mesh")
        to_value = lambda s: 1.0 / (s * wl.ne / ne)
    elif isinstance(wl, BatchedWL):
        ks, sizes, boxes = wl.instances()
        wl.count = len(sizes) + len(boxes)
        wl.grad_bytes = (sum(8 * (int(n) * int(n) + 2 * int(n)) for n in sizes)
                         + sum(6 * a * b * c * (16 + 96) + 2 * (a + 1) * (b + 1) * (c + 1) * 8
                               for a, b, c in boxes))
        nd, nt = 16, min(2, len(boxes))  # the batch's 8 : 1 mix of dense and tet instances
        dense = [W.batched_dense_instance(ks[i], sizes[i]) for i in range(min(nd, len(ks)))]
        tets = [W.batched_tet_instance(k, boxes[k]) for k in range(nt)]

        def fn():
            for A, x in dense:
                O.quadform_grad(A, x)
            for mesh, u in tets:
                O.tet_grad(mesh.conn, mesh.G, u)

        sample = f"{nd} dense and {nt} tet instances of the batch (its 8:1 mix) per step"
        to_value = lambda s: (nd + nt) / s
    elif isinstance(wl, HvpWL):
        mesh, u = W.tet_inputs(wl.a)
        wl.mesh, wl.u_host, wl.ne, wl.nv = mesh, u, mesh.ne, mesh.nv
        ne = min(mesh.ne, 500_000)
        conn, G = mesh.conn[:ne], mesh.G[:ne]
        v = np.random.default_rng(43).uniform(-1.0, 1.0, mesh.nv)
        unit_bytes = ne * (16 + 12 * wl.es) + 3 * mesh.nv * wl.es
        fn = lambda: O.tet_hvp(conn, G, u, v)
        sample = f"Hessian-vector product on the first {ne} tets of the {wl.a}^3 mesh per step"
        to_value = lambda s: unit_bytes / 1e9 / s
    elif isinstance(wl, TetWL):
        mesh, u = W.tet_inputs(wl.a)
        wl.mesh, wl.u_host, wl.ne, wl.nv = mesh, u, mesh.ne, mesh.nv
        G = mesh.G if wl.dtype == "f64" else mesh.G.astype("float32").astype("float64")
        if wl.dtype == "f32":
            u = u.astype("float32").astype("float64")
        try:
            cores = O.omp_threads()
            conn = mesh.conn
            unit_bytes = mesh.ne * (16 + 12 * wl.es) + 2 * mesh.nv * wl.es
            fn = lambda: O.tet_grad_omp(conn, G, u)
            sample = (f"full value+grad of the {wl.a}^3 mesh ({mesh.ne} tets) per step (oracle, "
                      f"OpenMP build, {cores} threads)")
        except Exception:  # noqa: BLE001  (no OpenMP build: serial oracle on 500k tets)
            ne = min(mesh.ne, 500_000)
            conn, G = mesh.conn[:ne], G[:ne]
            unit_bytes = ne * (16 + 12 * wl.es) + 2 * mesh.nv * wl.es
            fn = lambda: O.tet_grad(conn, G, u)
            sample = f"value+grad of the first {ne} tets of the {wl.a}^3 mesh per step"
        to_value = lambda s: unit_bytes / 1e9 / s
    elif isinstance(wl, SparseWL):
        A, x = W.spquadform_inputs(wl.m)
        if wl.dtype == "f32":
            A.val = A.val.astype("float32").astype("float64")
            x = x.astype("float32").astype("float64")
        wl.A, wl.n, wl.nnz = A, A.n, A.nnz
        fn = lambda: O.spquadform_grad(A.rowptr, A.col, A.val, x)
        sample = f"one full value+grad of the {A.m}x{A.n} CSR problem per step"
        to_value = lambda s: wl.grad_bytes / 1e9 / s
    elif isinstance(wl, LaplaceWL):
        x, b = W.laplace1d_inputs(wl.n)
        fn = lambda: O.laplace1d_grad(x, b)
        sample = f"one value+grad at n={wl.n} per step"
        to_value = lambda s: 1.0 / s
    else:
        raise SystemExit(f"no oracle reference for workload {args.workload}")
    for _ in range(args.warmup):
        fn()
    K = args.steps if args.steps > 0 else 10
    t0 = time.perf_counter()
    for _ in range(K):
        fn()
    s = (time.perf_counter() - t0) / K
    v = to_value(s)
    out = {"metric": METRIC, "value": round(v, 5), "unit": wl.unit, "n_gpus": world, "steps": K,
           "warmup": args.warmup, "ms_per_step": round(s * 1e3, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": wl.dtype_name,
           "data": "synthetic (seeded numpy PCG64 draws)", "config": wl.config(),
           "impl": "reference",
           "cpu_baseline": {"value": round(v, 5), "unit": wl.unit, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(v, 5), "unit": wl.unit, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
