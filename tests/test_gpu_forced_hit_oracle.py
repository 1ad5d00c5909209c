"""Forced isotropic turbulence on a 64^3 periodic box (Sec. II.C spectral force with the
Kupershtokh source of Sec. II.A) over its first 1000 steps, every form against the FP64
oracle's kinetic-energy curve and energy spectra of its operator
(tests/golden/hit64_forced_{bgk,nco}.txt, written by tests/golden/make_hit64_forced.py from
oracle/ alone). The chaotic flow is followed for 1000 steps, about two and a half turnover
times of its energetic eddies, so FP32 rounding is amplified only moderately and the curves
can still be compared point by point.

Bounds: the FP32 forms (FP32 storage with the FP32 CUDA-core or the split-BF16 tensor-core
network, FP32 BGK) keep k within 1e-4 of the oracle, the bound of the 1000-step FP32
parity run at 16^3; the forms with the BF16 tensor-core network (on FP16 f - w or FP32
storage) and FP16 BGK within 1e-3, the bound stated for the mixed form. The spectra every 100 steps
must agree within ten times the form's k bound in relative L1 over the energy-holding shells
1..32. The same run without the force misses the k bound by more than a hundred times (the
last test), so the comparison sees the forcing, not only the decay.
"""

import os
import re

import numpy as np
import pytest

import lbm_inputs
import paper_2412_08229_gb300 as P
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
N, NU, EVERY = 64, 0.0015, 10
FORMS = {  # name: (operator, storage, network, k bound)
    "bgk_f32": ("bgk", "f32", "f32", 1e-4),
    "nco_fp32": ("nco", "f32", "f32", 1e-4),
    "nco_split_bf16": ("nco", "f32", "bf16x3", 1e-4),
    "bgk_f16": ("bgk", "f16", "f32", 1e-3),
    "nco_mixed": ("nco", "f16", "bf16", 1e-3),
    "nco_bf16_f32_storage": ("nco", "f32", "bf16", 1e-3),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P._abi.load()


def _golden(op):
    path = os.path.join(GOLDEN, f"hit64_forced_{op}.txt")
    if not os.path.exists(path):
        pytest.skip(f"{os.path.basename(path)} has not been written (tests/golden/make_hit64_forced.py {op})")
    power, ks, es = None, [], {}
    for ln in open(path):
        m = re.search(r"power = ([0-9.eE+-]+)", ln)
        if ln.startswith("#"):
            if m:
                power = float(m.group(1))
            continue
        f = ln.split()
        if f[0] == "k":
            ks.append((int(f[1]), float(f[2])))
        elif f[0] == "E":
            es[int(f[1])] = np.array([float(v) for v in f[2:]])
    return power, np.array(ks), es


@pytest.mark.parametrize("form", sorted(FORMS))
def test_forced_hit64_against_the_oracle_over_1000_steps(form):
    op, storage, net, kbound = FORMS[form]
    power, ks, es = _golden(op)
    ctx = G.make_ctx((N, N, N), NU, op, storage=storage, net=net, theta=G.theta0() if op == "nco" else None,
                     forcing=dict(power=power))
    rho, u = lbm_inputs.isotropic_field(N, 1, 0.04)
    G.init_gpu(ctx, rho, u)
    steps = int(ks[-1, 0])
    phi, psi = lbm_inputs.forcing_draws(steps, seed=1)
    P.lbm_force_draws(ctx, phi, psi)
    ke = [P.lbm_kinetic_energy(ctx)]
    spectra = {}
    for t in range(0, steps + 1, EVERY):
        if t > 0:
            P.lbm_step(ctx, EVERY)
            ke.append(P.lbm_kinetic_energy(ctx))
        if t in es:
            E = torch.zeros(len(es[t]), dtype=torch.float64, device="cuda")
            P.lbm_energy_spectrum(ctx, E)
            spectra[t] = E.cpu().numpy()
    assert P.lbm_check(ctx) == 0
    P.lbm_destroy(ctx)
    k = np.array(ke)
    kerr = float(np.max(np.abs(k - ks[:, 1]) / ks[:, 1]))
    assert kerr <= kbound, kerr
    for t, Eo in es.items():
        sh = np.arange(1, min(33, len(Eo)))
        sh = sh[Eo[sh] > 1e-10 * Eo.sum()]
        l1 = float(np.sum(np.abs(spectra[t][sh] - Eo[sh])) / np.sum(Eo[sh]))
        assert l1 <= 10 * kbound, (t, l1)


def test_the_bound_rejects_the_unforced_run():
    """FP32 BGK on the same field without the force, against the forced oracle curve: k
    leaves the FP32 bound by more than a factor 100."""
    _, ks, _ = _golden("bgk")
    ctx = G.make_ctx((N, N, N), NU, "bgk")
    rho, u = lbm_inputs.isotropic_field(N, 1, 0.04)
    G.init_gpu(ctx, rho, u)
    ke = [P.lbm_kinetic_energy(ctx)]
    for _ in range(int(ks[-1, 0]) // EVERY):
        P.lbm_step(ctx, EVERY)
        ke.append(P.lbm_kinetic_energy(ctx))
    P.lbm_destroy(ctx)
    kerr = float(np.max(np.abs(np.array(ke) - ks[:, 1]) / ks[:, 1]))
    assert kerr > 100 * FORMS["bgk_f32"][3], kerr
