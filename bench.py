#!/usr/bin/env python
"""Benchmark: D3Q27 neural-collision (NCO) step throughput at 256^3 on GB300.

Workload: the 3-D Taylor-Green vortex at 256^3, Re 1600 (nu = 0.05 * 256 / (2 pi 1600)),
U0 = 0.05, rho = 1, NCO with Kaiming-uniform seed-0 weights. One "step" is one fused
pull-stream-collide kernel over the whole grid. Forms:
  fp32     - FP32 populations, FP32 network on CUDA cores;
  fp32_tc3 - FP32 populations, split-BF16 network on the tcgen05 tensor cores (three
             products per BF16 pair, FP32 accumulation: FP32-class network);
  fp32_tc  - FP32 populations, BF16 network on the tensor cores;
  mixed    - FP16 populations stored as f - w, BF16 network on the tensor cores.
The state (1.8 GB FP32, 0.9 GB FP16) is far larger than the 129 MB L2, so no flush is
needed between steps.

`--impl reference` times the FP64 CPU oracle (the only reference this method has) on
the machine's host cores, on a bounded slab sample of the same workload.
"""

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

NCORES = len(os.sched_getaffinity(0))
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, str(NCORES))

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3Q27 neural-collision MLUPS @256^3, % HBM roofline, mixed vs FP32 at stated error"
BYTES_PER_CELL = {"f32": 216, "f16": 108, "bf16": 108}  # 27 reads + 27 writes per cell-update
# network work per cell-update. Algorithmic: 47,920 flop, the exact folds of the group
# average (layer 3 after the group mean, layer 1 as 6 axis permutations x an 8-point
# Walsh-Hadamard transform over the sign flips: 6 x 540 MAC + 6 x 20 x 24 adds, layer 2
# 48 x 400 MAC). Useful as evaluated: 48 x (27 x 20 + 20 x 20) MAC (layer 1 per element).
# Issued on the tensor pipe with K and N padded: the pair kernel (two-layer BF16 network)
# runs 24 pairs x (K 32 x N 48 + K 48 x N 48) = 92,160 MAC per cell; the split-BF16 kernel
# 3 x (12 chunks x (K 32 x N 80) + 48 elements x (K 32 x N 32)) = 3 x 79,872.
ALGO_FLOPS_PER_CELL = 2 * (6 * 540 + 48 * 400) + 6 * 20 * 24 + 2 * 4 * 20
NET_FLOPS_PER_CELL = 2 * 48 * (27 * 20 + 20 * 20)
MMA_FLOPS_PER_CELL = {"bf16": 2 * 92160, "bf16x3": 3 * 2 * 79872}
N = 256
U0 = 0.05
RE = 1600.0
# DRAM bytes per 256^3 launch of each form's step kernel (dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture of that launch), or absent. Must be retaken (or
# removed) whenever the kernel changes.
TRAFFIC_256 = {
    "mixed": (907.16e6 + 865.96e6,
              "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none -k regex:nco_tcp "
              "-s 1 -c 1 python bench.py --forms mixed --steps 2 --warmup 1 --no-cpu --no-e2e --no-extras "
              "(one pass): 907.16 + 865.96 MB"),
}


def max_over_ranks(value):
    """The largest of one float per rank (every rank gets it); the value itself when no
    process group is running. NCCL reduces on the current GPU, gloo on the host."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(cells_per_rank, ms_max, world):
    """Whole-job throughput of `world` replicas that each update cells_per_rank cells per
    step, timed by the slowest replica (weak scaling)."""
    return cells_per_rank * world / (ms_max * 1e-3) / 1e6


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 1900.0, 2070.0, "fallback"


def tgv_slab(n, z0, nz, u0):
    """Taylor-Green fields on z-slab [z0, z0+nz) of the n^3 periodic grid (SoA, float64)."""
    import lbm_inputs
    x = lbm_inputs.grid_coordinates(n)
    z = x[z0:z0 + nz]
    Z, Y, X = np.meshgrid(z, x, x, indexing="ij")
    u = np.stack([u0 * np.sin(X) * np.cos(Y) * np.cos(Z), -u0 * np.cos(X) * np.sin(Y) * np.cos(Z),
                  np.zeros_like(X)])
    return np.ones((nz, n, n)), u


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[3:7]):
                if flag.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


FORMS = {
    # name: (operator, storage, network precision)
    "fp32": ("nco", "f32", "f32"),
    "mixed": ("nco", "f16", "bf16"),
    "fp32_tc": ("nco", "f32", "bf16"),
    "fp32_tc3": ("nco", "f32", "bf16x3"),
    "bgk_f32": ("bgk", "f32", "f32"),
    "kbc_f32": ("kbc", "f32", "f32"),
    "bgk_f16": ("bgk", "f16", "f32"),
    "kbc_f16": ("kbc", "f16", "f32"),
    "reg_f32": ("reg", "f32", "f32"),
}


def make_ctx(P, torch, form, n, nu, theta):
    op, storage, net = FORMS[form]
    ctx = P.lbm_create(n, n, n, nu, op=op, storage=storage, net=net)
    if op == "nco":
        P.nco_set_weights(ctx, torch.from_numpy(theta).cuda())
    return ctx, storage


def device_fields(torch, n, u0):
    import lbm_inputs
    rho, u = lbm_inputs.taylor_green_3d(n, u0)
    return (torch.from_numpy(rho.astype(np.float32)).cuda(), torch.from_numpy(u.astype(np.float32)).cuda())


def time_form(P, torch, form, n, nu, theta, steps, warmup, fields, barrier):
    ctx, storage = make_ctx(P, torch, form, n, nu, theta)
    P.lbm_init(ctx, *fields)
    P.lbm_step(ctx, warmup)
    torch.cuda.synchronize()
    barrier()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    P.lbm_step(ctx, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / steps
    status = P.lbm_check(ctx)
    del ctx
    return ms, storage, status


def time_e2e(P, torch, form, n, nu, theta, steps, barrier, repeats=3):
    """Same metric through the public API with host buffers: upload the initial fields
    from pinned host memory, then every step read the kinetic energy back to the host.
    The timed region runs `repeats` times; the median is reported (one host-side stall
    of a shared box otherwise decides the number)."""
    import lbm_inputs
    rho, u = lbm_inputs.taylor_green_3d(n, U0)
    rho_h = torch.from_numpy(rho.astype(np.float32)).pin_memory()
    u_h = torch.from_numpy(u.astype(np.float32)).pin_memory()
    ke_h = torch.zeros(1, dtype=torch.float64).pin_memory()
    ctx, storage = make_ctx(P, torch, form, n, nu, theta)
    P.lbm_init(ctx, rho_h, u_h)  # warm the staging path
    P.lbm_step(ctx, 2)
    torch.cuda.synchronize()
    times = []
    for _ in range(repeats):
        barrier()
        t0 = time.perf_counter()
        P.lbm_init(ctx, rho_h, u_h)
        for _ in range(steps):
            P.lbm_step(ctx, 1)
            P.lbm_kinetic_energy(ctx, ke_h)
        torch.cuda.synchronize()
        times.append(max_over_ranks(time.perf_counter() - t0))
    barrier()
    del ctx
    cells = n ** 3
    return {"seconds": float(np.median(times)), "all_seconds": [round(t, 5) for t in times],
            "h2d_bytes_per_step": int(16 * cells / steps), "d2h_bytes_per_step": 8}


def oracle_mlups(n, nu, theta, budget_s):
    """Time the FP64 oracle NCO step on z-slabs of the n^3 workload until budget_s is spent."""
    from oracle import collision as col
    from oracle import stepper as S
    nz = 2
    rho, u = tgv_slab(n, 0, nz, U0)
    sim = S.Simulation.from_macroscopic(rho, np.moveaxis(u, 0, -1), col.tau_from_nu(nu), op="nco",
                                        theta=theta.astype(np.float64))
    cells, t = 0, 0.0
    while t < budget_s:
        t0 = time.perf_counter()
        sim.step(1)
        t += time.perf_counter() - t0
        cells += n * n * nz
    return cells / t / 1e6, f"{cells // (n * n * nz)} oracle NCO steps on a {n}x{n}x{nz} z-slab of the {n}^3 TGV", t


def _torch_spectrum(torch, u, nbins):
    """E(n) of a (3, nz, ny, nx) velocity tensor, nearest-integer shells (user-side loss code)."""
    nz, ny, nx = u.shape[1:]
    uh = torch.fft.fftn(u, dim=(1, 2, 3)) / (nx * ny * nz)
    e = 0.5 * (uh.real ** 2 + uh.imag ** 2).sum(0)
    k = [torch.fft.fftfreq(m, d=1.0 / m, device=u.device) for m in (nz, ny, nx)]
    KZ, KY, KX = torch.meshgrid(*k, indexing="ij")
    shell = torch.round(torch.sqrt(KX * KX + KY * KY + KZ * KZ)).long().clamp(max=nbins - 1)
    return torch.zeros(nbins, dtype=e.dtype, device=u.device).index_add(0, shell.reshape(-1), e.reshape(-1))


def _unfold(torch, u):
    out = u
    for ax, comp in ((3, 0), (2, 1), (1, 2)):
        m = torch.flip(out, dims=(ax,)).clone()
        m[comp] = -m[comp]
        out = torch.cat([out, m], dim=ax)
    return out


def differentiation_form(P, torch):
    """Config 3: one training step on the reduced Taylor-Green model.

    Octant [0, pi]^3 on 32^3 nodes with mirror planes (full box 64^3), Re 3000, 200
    unrolled steps recorded with a checkpoint every 20; loss = relative spectrum
    discrepancy over shells 2..16 + 20 E(32) against a 128^3 FP32 BGK run of the same
    flow at the same physical time (400 steps). Times the forward and nco_backward.
    """
    import lbm_inputs
    n, re, steps, k = 32, 3000.0, 200, 20
    nu = lbm_inputs.reynolds_viscosity(U0, 2 * n, re)
    # reference spectrum: the same flow on the full 128^3 box, FP32 BGK, same physical time
    nr = 128
    ref = P.lbm_create(nr, nr, nr, lbm_inputs.reynolds_viscosity(U0, nr, re), op="bgk")
    rho, u = lbm_inputs.taylor_green_3d(nr, U0, shifted=True)
    P.lbm_init(ref, torch.from_numpy(rho.astype(np.float32)).cuda(), torch.from_numpy(u.astype(np.float32)).cuda())
    P.lbm_step(ref, steps * nr // (2 * n))
    E_ref = torch.zeros(nr // 2 + 1, dtype=torch.float64, device="cuda")
    P.lbm_energy_spectrum(ref, E_ref)
    del ref
    theta = torch.from_numpy(lbm_inputs.nco_parameters(0).astype(np.float32)).cuda()
    ctx = P.lbm_create(n, n, n, nu, op="nco", boundary="mirror")
    P.nco_set_weights(ctx, theta)
    rho, u = lbm_inputs.taylor_green_octant(n, U0)
    rho_d = torch.from_numpy(rho.astype(np.float32)).cuda()
    u_d = torch.from_numpy(u.astype(np.float32)).cuda()
    _torch_spectrum(torch, torch.zeros((3, 2 * n, 2 * n, 2 * n), dtype=torch.float64, device="cuda"), n + 1)
    free0 = torch.cuda.mem_get_info()[0]  # FFT library loaded and planned above, outside the timing
    P.lbm_init(ctx, rho_d, u_d)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P.lbm_record_begin(ctx, k)
    P.lbm_step(ctx, steps)
    rho_o = torch.empty((n, n, n), device="cuda")
    u_o = torch.empty((3, n, n, n), device="cuda")
    P.lbm_macroscopic(ctx, rho_o, u_o)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    uu = u_o.double().requires_grad_(True)
    E = _torch_spectrum(torch, _unfold(torch, uu), n + 1)
    sl = slice(2, 17)
    rel = (E[sl] - E_ref[sl]) / E_ref[sl]
    loss = (rel * rel).mean() + 20.0 * E[n]
    loss.backward()
    du = uu.grad.float().contiguous()
    dtheta = torch.zeros(1064, device="cuda")
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    P.nco_backward(ctx, du, None, dtheta, None)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    free1 = torch.cuda.mem_get_info()[0]
    del ctx
    return {"config": "TGV octant 32^3 mirror planes, Re 3000, 200 steps, checkpoint every 20, "
                      "loss vs 128^3 FP32 BGK spectrum (shells 2..16 + 20 E(32))",
            "forward_s": round(t1 - t0, 4), "loss_s": round(t2 - t1, 4), "backward_s": round(t3 - t2, 4),
            "backward_over_forward": round((t3 - t2) / (t1 - t0), 2), "loss": float(loss.item()),
            "grad_norm": float(dtheta.norm().item()),
            "device_bytes_for_state_checkpoints_and_work": int(free0 - free1)}


def dissipation_training_form(P, torch):
    """One sample of the time-dependent training (Sec. IV): the reduced Taylor-Green domain
    [0, pi/2]^3 (Appendix A) on 16^3 nodes (full box 64^3), Re 1600, Ma 0.1, the
    three-hidden-layer network, k sampled 102 times over t in [0, 15] (t in L / U0), loss =
    MSE of -dk/dt at the 100 interior samples against a reference curve; forward
    (NCOKineticEnergyUnroll) and adjoint (nco_backward_ke) timed. The reference curve stands
    in for the paper's 512^3 DNS: the same flow on a 32^3 reduced domain (full 128^3),
    FP32 BGK, sampled at the same physical times."""
    import lbm_inputs
    from paper_2412_08229_gb300.autograd import NCOKineticEnergyUnroll, dissipation_mse
    n, re, ma, nsamp = 16, 1600.0, 0.1, 100
    u0 = ma / np.sqrt(3.0)

    def setup(nr, op, theta=None):
        nu = lbm_inputs.reynolds_viscosity(u0, 4 * nr, re)
        c = P.lbm_create(nr, nr, nr, nu, op=op, boundary="tgv_reduced")
        if theta is not None:
            P.nco_set_weights(c, theta)
        rho, u = lbm_inputs.taylor_green_3d(4 * nr, u0, shifted=True)
        P.lbm_init(c, torch.from_numpy(np.ascontiguousarray(rho[:nr, :nr, :nr], dtype=np.float32)).cuda(),
                   torch.from_numpy(np.ascontiguousarray(u[:, :nr, :nr, :nr], dtype=np.float32)).cuda())
        tc = 4 * nr / (2 * np.pi * u0)          # steps per unit of t = L / U0
        every = int(round(15.0 * tc / (nsamp + 1)))
        return c, every, every / tc

    ref, every_r, dt_r = setup(2 * n, "bgk")
    ke_r = torch.zeros(nsamp + 2, dtype=torch.float64, device="cuda")
    for j in range(nsamp + 2):
        if j:
            P.lbm_step(ref, every_r)
        P.lbm_kinetic_energy(ref, ke_r[j:j + 1])
    del ref
    ke_r = ke_r / u0 ** 2
    eps_ref = -(ke_r[2:] - ke_r[:-2]) / (2.0 * dt_r)

    theta = torch.from_numpy(lbm_inputs.nco_parameters(0, (27, 20, 20, 20, 4)).astype(np.float32)).cuda()
    ctx, every, dt = setup(n, "nco", theta)
    f0 = torch.empty((27, n, n, n), dtype=torch.float32, device="cuda")
    P.lbm_get_state(ctx, f0)
    obs = [every * j for j in range(nsamp + 2)]
    th = theta.clone().requires_grad_(True)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    t0 = time.perf_counter()
    ke = NCOKineticEnergyUnroll.apply(th, ctx, f0, obs, every)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss = dissipation_mse(ke / u0 ** 2, dt, eps_ref)
    loss.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    free1 = torch.cuda.mem_get_info()[0]
    status = P.lbm_check(ctx)
    del ctx
    state_bytes = n ** 3 * 27 * 4
    return {"config": f"reduced TGV {n}^3 (full {4 * n}^3), Re {re:.0f}, Ma {ma}, 27-20-20-20-4 network, "
                      f"{obs[-1]} steps (t in [0, 15]), k every {every} steps, checkpoint every {every}; "
                      f"reference: 32^3 reduced (full 128^3) FP32 BGK",
            "forward_s": round(t1 - t0, 4), "loss_and_backward_s": round(t2 - t1, 4),
            "backward_over_forward": round((t2 - t1) / (t1 - t0), 2), "loss": float(loss.item()),
            "grad_norm": float(th.grad.norm().item()), "unstable": status != 0,
            "state_bytes_reduced": state_bytes, "state_bytes_full_box": 64 * state_bytes,
            "device_bytes_for_checkpoints_and_work": int(free0 - free1)}


def dissipation_epoch_form(P, torch, t_end=3.0, nsamp=20):
    """The Re-1600 row of the paper's epoch of time-dependent training cases (Sec. IV,
    Table of training cases: reduced domains 16^3 at Ma 0.05; 10^3, 16^3, 25^3 at Ma 0.1;
    10^3 to 32^3 at Ma 0.15 and 0.2): one training sample per case (three-hidden-layer
    network, k sampled nsamp + 2 times over t in [0, t_end], loss = the dissipation MSE,
    forward and adjoint), first one case after another, then all side by side with one
    host thread and one CUDA stream per case. t_end = 3 instead of the paper's 15 keeps the
    measurement short; the reference curve is zero (a timing, not a training run)."""
    import threading
    import lbm_inputs
    re = 1600.0
    cases = [(0.05, 16), (0.1, 10), (0.1, 16), (0.1, 25), (0.15, 10), (0.15, 16), (0.15, 25), (0.15, 32),
             (0.2, 10), (0.2, 16), (0.2, 25), (0.2, 32)]
    theta = lbm_inputs.nco_parameters(0, (27, 20, 20, 20, 4)).astype(np.float32)
    errors = []

    def one_case(ma, n, stream):
        ctx = None
        try:
            with torch.cuda.stream(stream):
                u0 = ma / np.sqrt(3.0)
                nu = lbm_inputs.reynolds_viscosity(u0, 4 * n, re)
                ctx = P.lbm_create(n, n, n, nu, op="nco", boundary="tgv_reduced")
                P.nco_set_weights(ctx, torch.from_numpy(theta).cuda())
                rho, u = lbm_inputs.taylor_green_3d(4 * n, u0, shifted=True)
                P.lbm_init(ctx, torch.from_numpy(np.ascontiguousarray(rho[:n, :n, :n], dtype=np.float32)).cuda(),
                           torch.from_numpy(np.ascontiguousarray(u[:, :n, :n, :n], dtype=np.float32)).cuda())
                tc = 4 * n / (2 * np.pi * u0)
                every = max(1, int(round(t_end * tc / (nsamp + 1))))
                obs = [every * j for j in range(nsamp + 2)]
                dt = every / tc
                # forward with kinetic-energy observations, then the loss's dL/dk in closed form
                # and the adjoint through the C ABI (no autograd engine between the threads)
                P.lbm_record_begin(ctx, every)
                ke = torch.empty(len(obs), dtype=torch.float64, device="cuda")
                P.lbm_kinetic_energy(ctx, ke[0:1])
                for j in range(1, len(obs)):
                    P.lbm_step(ctx, every)
                    P.lbm_kinetic_energy(ctx, ke[j:j + 1])
                k = ke.cpu().numpy() / u0 ** 2
                eps = -(k[2:] - k[:-2]) / (2.0 * dt)          # reference curve: zero
                g_eps = 2.0 * eps / eps.size
                dk = np.zeros_like(k)
                dk[2:] -= g_eps / (2.0 * dt)
                dk[:-2] += g_eps / (2.0 * dt)
                grad = torch.empty(theta.size, dtype=torch.float32, device="cuda")
                P.nco_backward_ke(ctx, obs, dk / u0 ** 2, dL_dtheta=grad)
                torch.cuda.current_stream().synchronize()
        except Exception as e:  # reported in the result, the other cases go on
            errors.append(f"{ma}/{n}: {e}")
        finally:
            if ctx is not None:
                stream.synchronize()
                P.lbm_destroy(ctx)

    one_case(0.1, 10, torch.cuda.current_stream())  # warm-up: library, pool and kernels loaded
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ma, n in cases:
        one_case(ma, n, torch.cuda.current_stream())
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    streams = [torch.cuda.Stream() for _ in cases]
    threads = [threading.Thread(target=one_case, args=(ma, n, st)) for (ma, n), st in zip(cases, streams)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    t_par = time.perf_counter() - t0
    return {"config": f"Re 1600 row of the training table: {len(cases)} reduced domains 10^3..32^3, Ma 0.05..0.2, "
                      f"27-20-20-20-4 network, t in [0, {t_end}], {nsamp + 2} k samples, forward + adjoint",
            "one_after_another_s": round(t_seq, 3), "side_by_side_s": round(t_par, 3),
            # a failed case shortens one arm: no speedup is claimed from unequal work
            "speedup": round(t_seq / t_par, 2) if not errors else None, "errors": errors}


def forced_training_form(P, torch, steps=200, k=20):
    """One training sample of the spectrum-loss procedure (Secs. II.D, III.A) on forced
    isotropic turbulence: 64^3, seed-1 field, u_rms 0.04, nu 0.0015, spectral forcing, NCO
    (FP32 storage and network), 200 recorded steps with a checkpoint every 20; loss = mean
    relative spectrum discrepancy over shells 4..10 + 20 E(32). The paper's reference is a
    DNS spectrum; the stand-in is the initial field's spectrum (the state the forcing is
    set to sustain). Times the forward, the loss and the adjoint through the forced steps."""
    import lbm_inputs
    n, nu = 64, 0.0015
    rho, u = lbm_inputs.isotropic_field(n, 1, 0.04)
    grads = [np.gradient(u[a], axis=ax) for a in range(3) for ax in range(3)]
    power = float(nu * np.mean(sum(g * g for g in grads)))
    phi, psi = lbm_inputs.forcing_draws(steps, seed=1)
    theta = torch.from_numpy(lbm_inputs.nco_parameters(0).astype(np.float32)).cuda()
    ctx = P.lbm_create(n, n, n, nu, op="nco", forcing=dict(power=power))
    P.nco_set_weights(ctx, theta)
    u0 = torch.from_numpy(u.astype(np.float32)).cuda()
    P.lbm_init(ctx, torch.from_numpy(rho.astype(np.float32)).cuda(), u0)
    E_ref = _torch_spectrum(torch, u0.double(), n // 2 + 1).detach()
    P.lbm_force_draws(ctx, phi, psi)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    t0 = time.perf_counter()
    P.lbm_record_begin(ctx, k)
    P.lbm_step(ctx, steps)
    u_o = torch.empty((3, n, n, n), device="cuda")
    P.lbm_macroscopic(ctx, None, u_o)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    uu = u_o.double().requires_grad_(True)
    E = _torch_spectrum(torch, uu, n // 2 + 1)
    sl = slice(4, 11)
    rel = (E[sl] - E_ref[sl]) / E_ref[sl]
    loss = (rel * rel).mean() + 20.0 * E[n // 2]
    loss.backward()
    du = uu.grad.float().contiguous()
    dtheta = torch.zeros(1064, device="cuda")
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    P.nco_backward(ctx, du, None, dtheta, None)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    free1 = torch.cuda.mem_get_info()[0]
    status = P.lbm_check(ctx)
    del ctx
    return {"config": f"HIT 64^3 forced (P = {power:.3e}), NCO FP32, {steps} steps, checkpoint every {k}, "
                      "loss: shells 4..10 relative to the initial spectrum + 20 E(32)",
            "forward_s": round(t1 - t0, 4), "loss_s": round(t2 - t1, 4), "backward_s": round(t3 - t2, 4),
            "backward_over_forward": round((t3 - t2) / (t1 - t0), 2), "loss": float(loss.item()),
            "grad_norm": float(dtheta.norm().item()), "unstable": status != 0,
            "device_bytes_for_checkpoints_and_work": int(free0 - free1)}


def forced_turbulence(P, torch, steps=200):
    """Config 1 throughput: forced isotropic turbulence 64^3 (spectral forcing each step),
    NCO (mixed and FP32 storage with the BF16 network), BGK and KBC, plus the spectrum; each
    form also unforced on the same field (the cost of the forcing is the difference). A
    forced step is two launches: the coefficient kernel and the step kernel, which
    synthesises the force and projects the velocity in place."""
    import lbm_inputs
    n = 64
    nu = 0.0015
    rho, u = lbm_inputs.isotropic_field(n, 1, 0.04)
    # power input: the initial viscous dissipation nu <|grad u|^2> (lattice units)
    grads = [np.gradient(u[a], axis=ax) for a in range(3) for ax in range(3)]
    power = float(nu * np.mean(sum(g * g for g in grads)))
    phi, psi = lbm_inputs.forcing_draws(steps + 10, seed=1)
    theta = torch.from_numpy(lbm_inputs.nco_parameters(0).astype(np.float32)).cuda()
    out = {"config": f"HIT 64^3, seed 1, u_rms 0.04, nu 0.0015, forcing |k|<=2 with P = {power:.3e}", "forms": {}}
    for name, (op, storage, net) in {"nco_mixed": ("nco", "f16", "bf16"), "nco_fp32_tc": ("nco", "f32", "bf16"),
                                     "bgk_f32": ("bgk", "f32", "f32"), "kbc_f32": ("kbc", "f32", "f32")}.items():
        ctx = P.lbm_create(n, n, n, nu, op=op, storage=storage, net=net, forcing=dict(power=power))
        if op == "nco":
            P.nco_set_weights(ctx, theta)
        P.lbm_init(ctx, torch.from_numpy(rho.astype(np.float32)).cuda(), torch.from_numpy(u.astype(np.float32)).cuda())
        P.lbm_force_draws(ctx, phi, psi)
        P.lbm_step(ctx, 5)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        P.lbm_step(ctx, steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        E = torch.zeros(n // 2 + 1, dtype=torch.float64, device="cuda")
        e0.record()
        P.lbm_energy_spectrum(ctx, E)
        e1.record()
        torch.cuda.synchronize()
        out["forms"][name] = {"ms_per_step": round(ms, 4), "mlups": round(n ** 3 / (ms * 1e3), 1),
                              "spectrum_ms": round(e0.elapsed_time(e1), 4), "unstable": P.lbm_check(ctx) != 0}
        del ctx
        ctx = P.lbm_create(n, n, n, nu, op=op, storage=storage, net=net)
        if op == "nco":
            P.nco_set_weights(ctx, theta)
        P.lbm_init(ctx, torch.from_numpy(rho.astype(np.float32)).cuda(), torch.from_numpy(u.astype(np.float32)).cuda())
        P.lbm_step(ctx, 5)
        torch.cuda.synchronize()
        e0.record()
        P.lbm_step(ctx, steps)
        e1.record()
        torch.cuda.synchronize()
        out["forms"][name]["unforced_ms_per_step"] = round(e0.elapsed_time(e1) / steps, 4)
        del ctx
    return out


def batching_form(P, torch, steps=500, warmup=3):
    """Config 4: 48 independent NCO instances (F16 storage, BF16 network) of sizes drawn
    from {32, 48, 64, 96}^3 and Re log-uniform in [400, 20000] (seed 2), half Taylor-Green
    (U = 0.05) and half forced isotropic turbulence (u_rms = 0.04, seed-1 field, P = nu
    <|grad u|^2>), nu = U N / (2 pi Re). Stepped `steps` times by one persistent launch per
    step replayed from CUDA graphs with the autotuned tile shape, against the same
    instances stepped one after another with lbm_step."""
    import lbm_inputs
    rng = np.random.default_rng(2)
    count = 48
    sizes = rng.choice([32, 48, 64, 96], size=count)
    res = np.exp(rng.uniform(np.log(400.0), np.log(20000.0), size=count))
    theta = torch.from_numpy(lbm_inputs.nco_parameters(0).astype(np.float32)).cuda()
    specs, fields, draws = [], [], []
    hit_cache = {}
    for i in range(count):
        n, re, forced = int(sizes[i]), float(res[i]), i % 2 == 1
        u_ref = 0.04 if forced else U0
        nu = u_ref * n / (2.0 * np.pi * re)
        if forced:
            if n not in hit_cache:
                rho, u = lbm_inputs.isotropic_field(n, 1, 0.04)
                g2 = np.mean(sum(np.gradient(u[a], axis=ax) ** 2 for a in range(3) for ax in range(3)))
                hit_cache[n] = (rho, u, float(g2))
            rho, u, g2 = hit_cache[n]
            spec = dict(nx=n, ny=n, nz=n, nu=nu, storage="f16", forcing=dict(power=nu * g2))
            draws.append(lbm_inputs.forcing_draws(steps + 4 * warmup + 16, seed=100 + i))
        else:
            rho, u = lbm_inputs.taylor_green_3d(n, U0)
            spec = dict(nx=n, ny=n, nz=n, nu=nu, storage="f16")
            draws.append(None)
        specs.append(spec)
        fields.append((torch.from_numpy(rho.astype(np.float32)).cuda(), torch.from_numpy(u.astype(np.float32)).cuda()))
    cells = int(sum(int(n) ** 3 for n in sizes))

    def init(ctx, i):
        P.lbm_init(ctx, *fields[i])
        if draws[i] is not None:
            P.lbm_force_draws(ctx, *draws[i])

    out = {"config": f"{count} instances, sizes {{32,48,64,96}}^3, Re log-uniform [400, 20000] (seed 2), "
                     f"half TGV / half forced HIT, F16 storage, BF16 net, {steps} steps each",
           "cells": cells, "steps": steps}
    # batched: one persistent launch per step, replayed from CUDA graphs
    b = P.lbm_batch_create(specs)
    P.lbm_batch_set_weights(b, theta)
    for i in range(count):
        init(b[i], i)
    stream = torch.cuda.Stream()  # a timing stream; the batch runs on its own stream
    shape = P.lbm_batch_autotune(b)
    out["autotune_tile_shape"] = {0: "pairs of group elements across two warpgroups (2 tiles per SM)"}.get(
        shape, f"chunks of four group elements per warpgroup, {shape} warpgroups per SM")
    P.lbm_batch_step(b, warmup, use_graph=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P.lbm_batch_step(b, steps, use_graph=True)
    torch.cuda.synchronize()
    t_graph = time.perf_counter() - t0
    out["batched_graph"] = {"seconds": round(t_graph, 4), "mlups": round(cells * steps / t_graph / 1e6, 1),
                            "unstable_instances": int(sum(P.lbm_check(b[i]) != 0 for i in range(count)))}
    P.lbm_batch_step(b, 2, use_graph=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P.lbm_batch_step(b, 2 * warmup, use_graph=False)
    torch.cuda.synchronize()
    t_direct = (time.perf_counter() - t0) / (2 * warmup)
    out["batched_direct_ms_per_step"] = round(t_direct * 1e3, 3)
    del b, stream
    # sequential: every instance its own context, stepped on its own
    ctxs = []
    for i in range(count):
        sp = dict(specs[i])
        c = P.lbm_create(sp.pop("nx"), sp.pop("ny"), sp.pop("nz"), sp.pop("nu"), op="nco", net="bf16", **sp)
        P.nco_set_weights(c, theta)
        init(c, i)
        P.lbm_step(c, warmup)
        ctxs.append(c)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in ctxs:
        P.lbm_step(c, steps)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    out["sequential"] = {"seconds": round(t_seq, 4), "mlups": round(cells * steps / t_seq / 1e6, 1)}
    out["speedup_batched_over_sequential"] = round(t_seq / t_graph, 3)
    del ctxs
    return out


def _ke_curve(P, torch, form, n, nu, theta, steps, every, spectra_at=()):
    """k every `every` steps of the n^3 Re-1600 TGV in one form; the energy spectra at the
    steps in `spectra_at` (multiples of `every`), GPU FP64 bins."""
    import lbm_inputs
    op, storage, net = FORMS[form]
    ctx = P.lbm_create(n, n, n, nu, op=op, storage=storage, net=net)
    P.nco_set_weights(ctx, torch.from_numpy(theta).cuda())
    rho, u = lbm_inputs.taylor_green_3d(n, U0)
    P.lbm_init(ctx, torch.from_numpy(rho.astype(np.float32)).cuda(), torch.from_numpy(u.astype(np.float32)).cuda())
    ke = torch.zeros(steps // every + 1, dtype=torch.float64, device="cuda")
    spectra = {}
    P.lbm_kinetic_energy(ctx, ke[0:1])
    if 0 in spectra_at:
        spectra[0] = torch.zeros(spectra_at[0], dtype=torch.float64, device="cuda")
        P.lbm_energy_spectrum(ctx, spectra[0])
    for i in range(1, steps // every + 1):
        P.lbm_step(ctx, every)
        P.lbm_kinetic_energy(ctx, ke[i:i + 1])
        if i * every in spectra_at:
            E = torch.zeros(spectra_at[i * every], dtype=torch.float64, device="cuda")
            P.lbm_energy_spectrum(ctx, E)
            spectra[i * every] = E
    status = P.lbm_check(ctx)
    out = ke.cpu().numpy()
    spectra = {t: E.cpu().numpy() for t, E in spectra.items()}
    del ctx
    return out, status != 0, spectra


def _golden_rows(path):
    """(k rows, E rows) of a golden oracle file: 'step k' lines, or 'k step value' and
    'E step E(0) E(1) ...' lines."""
    ks, es = [], {}
    for ln in open(path):
        if not ln.strip() or ln.startswith("#"):
            continue
        f = ln.split()
        if f[0] == "k":
            ks.append((float(f[1]), float(f[2])))
        elif f[0] == "E":
            es[int(f[1])] = np.array([float(v) for v in f[2:]])
        else:
            ks.append((float(f[0]), float(f[1])))
    return np.array(ks), es


def _dissipation(k, every):
    return -(k[2:] - k[:-2]) / (2.0 * every)


def precision_form(P, torch):
    """Config 2 (precision): the Re-1600 TGV at 64^3 over 20 convective times (t_c =
    N / (2 pi U0) steps) in the mixed form (FP16 f - w storage, BF16 tensor-core network),
    the FP32-storage tensor-core forms (BF16 and split-BF16 network) and the FP32 form (FP32
    storage, FP32 CUDA-core network), each against the FP64 oracle's curve and spectra
    (tests/golden/tgv64_re1600_nco_20tc.txt, written by the oracle alone): the largest
    relative kinetic-energy error, the largest error of -dk/dt over the oracle's peak
    dissipation, and the spectrum error at the stored times (largest relative error over
    the shells 1..32 and the relative L1 error over them); and the forms against each other.
    At 256^3 over two convective times the tensor-core forms against each other (the
    split-BF16 form standing in for FP32; 20 convective times: the precision256 extra)."""
    import lbm_inputs
    theta = lbm_inputs.nco_parameters(0).astype(np.float32)
    out = {}
    n, every = 64, 10
    tc = n / (2 * math.pi * U0)
    nu = lbm_inputs.reynolds_viscosity(U0, n, RE)
    gpath = os.path.join(ROOT, "tests", "golden", "tgv64_re1600_nco_20tc.txt")
    g, gE = _golden_rows(gpath) if os.path.exists(gpath) else (None, {})
    steps = int(g[-1, 0]) if g is not None else int(round(20 * tc)) // every * every
    forms = ("fp32", "fp32_tc3", "mixed", "fp32_tc")
    curves, unstable, spectra = {}, {}, {}
    for form in forms:
        curves[form], unstable[form], spectra[form] = _ke_curve(
            P, torch, form, n, nu, theta, steps, every, {t: len(e) for t, e in gE.items()})
    ref = curves["fp32"]

    def rel_dev(a, b):
        return float(np.max(np.abs(a - b) / np.abs(b)))

    d_ref = _dissipation(ref, every)
    scale = float(np.max(np.abs(d_ref)))
    res64 = {"steps": steps, "convective_times": round(steps / tc, 2), "sample_every": every,
             "ke_final": {f: float(c[-1]) for f, c in curves.items()}, "unstable": unstable}
    for form in ("fp32_tc3", "mixed", "fp32_tc"):
        res64[f"{form}_vs_fp32_ke_max_rel"] = rel_dev(curves[form], ref)
        res64[f"{form}_vs_fp32_dissipation_max_abs_over_peak"] = float(
            np.max(np.abs(_dissipation(curves[form], every) - d_ref)) / scale)
    if g is not None:
        idx = (g[:, 0] / every).astype(int)
        d_o = _dissipation(g[:, 1], every)
        peak = float(np.max(np.abs(d_o)))
        vs = {}
        for form in forms:
            k = curves[form][idx]
            e = {"ke_max_rel": rel_dev(k, g[:, 1]),
                 "dissipation_max_abs_over_peak": float(np.max(np.abs(_dissipation(k, every) - d_o)) / peak)}
            for t, Eo in sorted(gE.items()):
                Eg = spectra[form][t][:len(Eo)]
                sh = np.arange(1, min(33, len(Eo)))
                sh = sh[Eo[sh] > 1e-10 * Eo.sum()]  # shells that hold energy (at t = 0 only shell 2)
                e[f"spectrum_t{t}_max_rel_shells_1_32"] = float(np.max(np.abs(Eg[sh] - Eo[sh]) / Eo[sh]))
                e[f"spectrum_t{t}_l1_rel_shells_1_32"] = float(np.sum(np.abs(Eg[sh] - Eo[sh])) / np.sum(Eo[sh]))
            vs[form] = e
        res64["vs_oracle"] = vs
        res64["oracle"] = {"file": os.path.relpath(gpath, ROOT), "steps": steps,
                           "spectrum_steps": sorted(gE), "dissipation_peak": peak}
    out["tgv64_re1600"] = res64
    out["hit64_forced"] = _hit64_forced_vs_oracle(P, torch)
    out["tgv256_re1600"] = _precision256(P, torch, theta, 2)
    return out


def _golden_power(path):
    """The forcing power recorded in a forced golden file's header ('power = <value>')."""
    import re
    for ln in open(path):
        m = re.search(r"power = ([0-9.eE+-]+)", ln)
        if m:
            return float(m.group(1))
    raise ValueError(f"no power in {path}")


def _hit64_forced_vs_oracle(P, torch):
    """Config 1 against the FP64 oracle: forced isotropic turbulence 64^3 (seed-1 field,
    u_rms 0.04, nu 0.0015, the spectral force with the draws of seed 1) over its first 1000
    steps, each form against the oracle's curve and spectra of its operator
    (tests/golden/hit64_forced_{bgk,nco}.txt, written by the oracle alone): the largest
    relative kinetic-energy error over the curve (every 10 steps) and the spectrum errors
    every 100 steps (largest relative error over the energy-holding shells 1..32 and the
    relative L1 error over them)."""
    import lbm_inputs
    n, nu, every = 64, 0.0015, 10
    rho, u = lbm_inputs.isotropic_field(n, 1, 0.04)
    theta = torch.from_numpy(lbm_inputs.nco_parameters(0).astype(np.float32)).cuda()
    out = {}
    for form, op_file in (("bgk_f32", "bgk"), ("bgk_f16", "bgk"), ("fp32", "nco"), ("fp32_tc3", "nco"),
                          ("mixed", "nco"), ("fp32_tc", "nco")):
        gpath = os.path.join(ROOT, "tests", "golden", f"hit64_forced_{op_file}.txt")
        if not os.path.exists(gpath):
            out[form] = {"skipped": f"{os.path.relpath(gpath, ROOT)} missing"}
            continue
        g, gE = _golden_rows(gpath)
        steps = int(g[-1, 0])
        op, storage, net = FORMS[form]
        ctx = P.lbm_create(n, n, n, nu, op=op, storage=storage, net=net, forcing=dict(power=_golden_power(gpath)))
        if op == "nco":
            P.nco_set_weights(ctx, theta)
        P.lbm_init(ctx, torch.from_numpy(rho.astype(np.float32)).cuda(), torch.from_numpy(u.astype(np.float32)).cuda())
        phi, psi = lbm_inputs.forcing_draws(steps, seed=1)
        P.lbm_force_draws(ctx, phi, psi)
        ke = torch.zeros(steps // every + 1, dtype=torch.float64, device="cuda")
        spectra = {}
        P.lbm_kinetic_energy(ctx, ke[0:1])
        for i in range(0, steps // every + 1):
            if i > 0:
                P.lbm_step(ctx, every)
                P.lbm_kinetic_energy(ctx, ke[i:i + 1])
            if i * every in gE:
                E = torch.zeros(len(gE[i * every]), dtype=torch.float64, device="cuda")
                P.lbm_energy_spectrum(ctx, E)
                spectra[i * every] = E
        unstable = P.lbm_check(ctx) != 0
        k = ke.cpu().numpy()[(g[:, 0] / every).astype(int)]
        e = {"ke_max_rel": float(np.max(np.abs(k - g[:, 1]) / g[:, 1])), "unstable": unstable,
             "oracle": os.path.relpath(gpath, ROOT)}
        for t, Eo in sorted(gE.items()):
            Eg = spectra[t].cpu().numpy()
            sh = np.arange(1, min(33, len(Eo)))
            sh = sh[Eo[sh] > 1e-10 * Eo.sum()]
            e[f"spectrum_t{t}_max_rel_shells_1_32"] = float(np.max(np.abs(Eg[sh] - Eo[sh]) / Eo[sh]))
            e[f"spectrum_t{t}_l1_rel_shells_1_32"] = float(np.sum(np.abs(Eg[sh] - Eo[sh])) / np.sum(Eo[sh]))
        out[form] = e
        del ctx
    return out


def _precision256(P, torch, theta, tcs):
    """The 256^3 Re-1600 TGV over `tcs` convective times: mixed and FP32-storage BF16 forms
    against the split-BF16 (FP32-class) form."""
    import lbm_inputs
    n, every = 256, 50
    tc = n / (2 * math.pi * U0)
    steps = int(round(tcs * tc)) // every * every
    nu = lbm_inputs.reynolds_viscosity(U0, n, RE)
    c_mixed, u1, _ = _ke_curve(P, torch, "mixed", n, nu, theta, steps, every)
    c_tc, u2, _ = _ke_curve(P, torch, "fp32_tc", n, nu, theta, steps, every)
    c_x3, u3, _ = _ke_curve(P, torch, "fp32_tc3", n, nu, theta, steps, every)

    def rel_dev(a, b):
        return float(np.max(np.abs(a - b) / np.abs(b)))

    res = {"steps": steps, "convective_times": round(steps / tc, 2), "sample_every": every,
           "mixed_vs_fp32_tc3_ke_max_rel": rel_dev(c_mixed, c_x3),
           "fp32_tc_vs_fp32_tc3_ke_max_rel": rel_dev(c_tc, c_x3),
           "mixed_vs_fp32_tc_ke_max_rel": rel_dev(c_mixed, c_tc), "ke_final_mixed": float(c_mixed[-1]),
           "unstable": {"mixed": u1, "fp32_tc": u2, "fp32_tc3": u3}}
    d3 = _dissipation(c_x3, every)
    sc = float(np.max(np.abs(d3)))
    res["mixed_vs_fp32_tc3_dissipation_max_abs_over_peak"] = float(np.max(np.abs(_dissipation(c_mixed, every) - d3)) / sc)
    res["fp32_tc_vs_fp32_tc3_dissipation_max_abs_over_peak"] = float(np.max(np.abs(_dissipation(c_tc, every) - d3)) / sc)
    return res


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle, as it stands, on the host cores. One timed step is
    one oracle NCO step on a z-slab (n x n x 2 cells) of the n^3 workload, so ms_per_step x
    steps is the time the arm spent; value = slab cells / median step time."""
    if rank != 0:
        return
    import lbm_inputs
    from oracle import collision as col
    from oracle import stepper as S
    theta = lbm_inputs.nco_parameters(0).astype(np.float32)
    n, nz = args.n, 2
    nu = lbm_inputs.reynolds_viscosity(U0, n, RE)
    rho, u = tgv_slab(n, 0, nz, U0)
    sim = S.Simulation.from_macroscopic(rho, np.moveaxis(u, 0, -1), col.tau_from_nu(nu), op="nco",
                                        theta=theta.astype(np.float64))
    for _ in range(args.warmup):
        sim.step(1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        sim.step(1)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.median(times))
    value = n * n * nz / (ms * 1e-3) / 1e6
    sample = f"one oracle NCO step on a {n}x{n}x{nz} z-slab ({n * n * nz} cells) of the {n}^3 TGV per timed step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"TGV {n}^3 Re1600, NCO (27-20-20-4, seed-0 Kaiming weights); each step: {sample}",
                   "n": n, "re": RE, "nu": nu, "slab_cells": n * n * nz, "parallelism": "rank 0 only"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": NCORES, "kind": "oracle", "sample": sample,
                         "seconds": round(float(np.sum(times)), 2)},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


_ORACLE_PROBE = """
import sys, time, numpy as np
sys.path.insert(0, {root!r})
import lbm_inputs
from oracle import collision as col, stepper as S
n = {n}
rho, u = lbm_inputs.taylor_green_3d(n, 0.05)
th = lbm_inputs.nco_parameters(0).astype(np.float32).astype(np.float64)
sim = S.Simulation.from_macroscopic(rho, np.moveaxis(u, 0, -1), col.tau_from_nu(0.005), op="nco", theta=th)
sim.step(1)
t0 = time.perf_counter(); sim.step({steps}); t = time.perf_counter() - t0
print(n ** 3 * {steps} / t / 1e6)
"""


def oracle_grid_timings():
    """The oracle NCO step at 16^3 and 64^3 (Taylor-Green), single-threaded and with every
    core this job owns, each in a fresh process so that the BLAS thread count is set before
    numpy loads. Returns {grid: {"1": MLUPS, str(NCORES): MLUPS}}."""
    out = {}
    for n, steps in ((16, 5), (64, 1)):
        row = {}
        for threads in sorted({1, NCORES}):
            env = dict(os.environ, OPENBLAS_NUM_THREADS=str(threads), OMP_NUM_THREADS=str(threads),
                       MKL_NUM_THREADS=str(threads))
            code = _ORACLE_PROBE.format(root=ROOT, n=n, steps=steps)
            r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
            row[f"{threads}_threads"] = float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
        out[f"{n}^3"] = row
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--forms", default="mixed,fp32_tc,fp32_tc3,fp32,bgk_f32,kbc_f32,bgk_f16")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the config 1-4 measurements")
    ap.add_argument("--extras", default="", help="comma-separated subset of the extra measurements (default: all)")
    ap.add_argument("--batch-steps", type=int, default=500, help="steps of every instance in the batching form")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import lbm_inputs
    import paper_2412_08229_gb300 as P

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        barrier = lambda: dist.barrier()  # noqa: E731
    else:
        barrier = lambda: None  # noqa: E731

    P._abi.load()
    n = args.n
    nu = lbm_inputs.reynolds_viscosity(U0, n, RE)
    theta = lbm_inputs.nco_parameters(0).astype(np.float32)
    fields = device_fields(torch, n, U0)
    hbm, bf16_tf, sm_max, peak_kind = peaks()

    forms = {}
    clocks = None
    for form in [f for f in args.forms.split(",") if f]:
        try:
            with ClockSampler(local) as cs:
                ms, storage, status = time_form(P, torch, form, n, nu, theta, args.steps, args.warmup, fields, barrier)
            clk = cs.summary()
        except P.LbmError as e:
            forms[form] = {"unavailable": str(e)}
            continue
        ms = max_over_ranks(ms)  # the slowest replica sets the time
        mlups = n ** 3 / (ms * 1e-3) / 1e6
        achieved = BYTES_PER_CELL[storage] * n ** 3 / (ms * 1e-3) / 1e9
        forms[form] = {"mlups": aggregate_mlups(n ** 3, ms, world), "mlups_per_gpu": mlups, "ms_per_step": ms, "storage": storage,
                       "hbm_gbs_algorithmic": achieved, "hbm_frac_of_measured": achieved / hbm,
                       "fp32_roofline_frac": mlups / (hbm * 1e9 / 216 / 1e6), "unstable": status != 0,
                       "clocks": clk}
        clocks = clk
    ok = {k: v for k, v in forms.items() if "mlups" in v}
    if not ok:
        raise SystemExit("no form could be timed: " + json.dumps(forms))
    nco_ok = [k for k in ("mixed", "fp32_tc", "fp32") if k in ok]
    head = nco_ok[0] if nco_ok else next(iter(ok))
    h = ok[head]

    e2e = None
    if not args.no_e2e:
        try:
            r = time_e2e(P, torch, head, n, nu, theta, max(args.steps, 5), barrier)
            e2e = {"value": n ** 3 * max(args.steps, 5) / r["seconds"] / 1e6 * world, "unit": "MLUPS",
                   "h2d_bytes_per_step": r["h2d_bytes_per_step"], "d2h_bytes_per_step": r["d2h_bytes_per_step"],
                   "note": "lbm_init from pinned host rho,u once, then per step lbm_step + KE read to host; "
                           "median of 3 timed repetitions", "repetitions_s": r["all_seconds"]}
        except P.LbmError as e:
            e2e = {"unavailable": str(e)}

    extras = {}
    if rank == 0 and not args.no_extras:
        runs = {"differentiation": lambda: differentiation_form(P, torch),
                "forced_turbulence": lambda: forced_turbulence(P, torch),
                "dissipation_training": lambda: dissipation_training_form(P, torch),
                "forced_training": lambda: forced_training_form(P, torch),
                "dissipation_epoch": lambda: dissipation_epoch_form(P, torch),
                "batching": lambda: batching_form(P, torch, steps=args.batch_steps),
                "precision": lambda: precision_form(P, torch),
                "precision256": lambda: {"tgv256_re1600_20tc": _precision256(
                    P, torch, lbm_inputs.nco_parameters(0).astype(np.float32), 20)}}
        default = [e for e in runs if e != "precision256"]  # minutes of 256^3 stepping: on request only
        chosen = [e for e in args.extras.split(",") if e] if args.extras else default
        for name in chosen:
            if name not in runs:
                raise SystemExit(f"unknown extra {name!r}; choose from {', '.join(runs)}")
            try:
                extras[name] = runs[name]()
            except P.LbmError as e:
                extras[name] = {"unavailable": str(e)}

    cpu = None
    if rank == 0 and not args.no_cpu:
        v, sample, secs = oracle_mlups(N, lbm_inputs.reynolds_viscosity(U0, N, RE), theta, 10.0)
        cpu = {"value": v, "unit": "MLUPS", "cores": NCORES, "kind": "oracle", "sample": sample,
               "seconds": round(secs, 2), "mlups_by_grid_and_threads": oracle_grid_timings()}

    if rank != 0:
        return
    traffic = TRAFFIC_256.get(head) if n == 256 else None
    hbm_view = {"achieved": h["hbm_gbs_algorithmic"], "peak": hbm, "unit": "GB/s",
                "frac": h["hbm_gbs_algorithmic"] / hbm,
                "peak_source": f"{peak_kind} MEASURED_PEAKS.json hbm_gbs (copy bandwidth)",
                "algorithmic_bytes_per_cell": BYTES_PER_CELL[h["storage"]]}
    net = FORMS[head][2]
    if net in MMA_FLOPS_PER_CELL:
        # the NCO's intensity (network flops per byte) lies far above the BF16 ridge: the
        # tensor roof binds it; achieved = algorithmic flops of one launch / its duration
        cells_per_s = n ** 3 / (h["ms_per_step"] * 1e-3)
        algo = ALGO_FLOPS_PER_CELL * cells_per_s / 1e12
        roof = {"bound": "tensor", "achieved": algo, "peak": bf16_tf, "unit": "TFLOP/s", "frac": algo / bf16_tf,
                "traffic": traffic[0] if traffic else None, "traffic_source": traffic[1] if traffic else None,
                "kernel": "fused pull-stream-collide step (one launch per step)",
                "peak_source": f"{peak_kind} MEASURED_PEAKS.json bf16_tflops (cuBLAS burst)",
                "algorithmic_flops_per_cell": ALGO_FLOPS_PER_CELL,
                "useful_flops_per_cell": NET_FLOPS_PER_CELL,
                "achieved_useful": NET_FLOPS_PER_CELL * cells_per_s / 1e12,
                "frac_useful": NET_FLOPS_PER_CELL * cells_per_s / 1e12 / bf16_tf,
                "mma_flops_per_cell": MMA_FLOPS_PER_CELL[net],
                "achieved_mma": MMA_FLOPS_PER_CELL[net] * cells_per_s / 1e12,
                "frac_mma": MMA_FLOPS_PER_CELL[net] * cells_per_s / 1e12 / bf16_tf,
                "hbm": hbm_view}
    else:
        roof = {"bound": "hbm", **{k: hbm_view[k] for k in ("achieved", "peak", "unit", "frac")},
                "traffic": traffic[0] if traffic else None, "traffic_source": traffic[1] if traffic else None,
                "kernel": "fused pull-stream-collide step (one launch per step)",
                "peak_source": hbm_view["peak_source"],
                "algorithmic_bytes_per_cell": hbm_view["algorithmic_bytes_per_cell"]}
    line = {
        "metric": METRIC, "value": h["mlups"], "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "f32", "mixed": "f32 collision, f16 storage, bf16 net",
                  "fp32_tc": "f32 collision and storage, bf16 net"}.get(head, head),
        "data": "synthetic",
        "config": {"workload": f"TGV {n}^3 Re1600 NCO (27-20-20-4, seed-0 Kaiming weights), form={head}",
                   "n": n, "re": RE, "nu": nu, "u0": U0, "parallelism": f"replicas x{world}",
                   "l2": "state larger than L2 (no flush needed)"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
        "clocks": clocks, "forms": forms, **extras,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
