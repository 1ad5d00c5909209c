"""Reference and tolerance of the BF16 tensor-core network (test infrastructure).

The tensor-core kernels evaluate the hidden layers of the invariant network (Sec. II.B,
eq. gconv_m) with BF16 operands and FP32 accumulation: the moment inputs, the weights and
biases of every hidden layer and every hidden activation that enters the next hidden layer
are rounded to BF16 (nearest even); the output layer runs in FP32 on the group sum of the
last hidden activations. The reference is the FP64 oracle evaluated with the same operand
rounding (oracle.collision.phi_network, operand_round=bf16).

What may still separate the kernel from that reference, and the bound taken for each:
  * an input moment whose FP32 value rounds to the other BF16 neighbour than its FP64
    value (both lie within a few FP32 ulps of a BF16 rounding boundary): first order in
    the network's Jacobian at the cell, |d tau~/d m_k| x ulp_bf16(m_k), for the two largest
    such terms (rounding boundaries are rarely met twice in one cell);
  * the same for a hidden activation after the FP32 accumulation: four times the largest
    |d tau~/d h| x ulp_bf16(h) over the cell's 48 x 20 activations of each rounded layer;
  * FP32 accumulation: 1e-6 + 1e-5 x (1/48) sum_g |W_out| relu(z_last) on tau~.
Twice that sum bounds |d tau~| (the factor covers ReLU kinks met by a flip), and
|d omega / d tau~| <= 1/2 (tau = 1/(2(1 + e^tau~)) + 1/2, Sec. II.B) turns it into a
bound on every learned rate. A rate error d omega_n moves the post-collision populations
by d omega_n M^-1 (m restricted to order n + 3), since m^eq has no moment above order 2.

The check of a step compares stored values: the kernel's stored deviation f - w must be
a rounding, in the storage format, of some value within the bound (plus 1e-5 max|f| of
FP32 arithmetic) of the reference. tests/test_bf16_tolerance.py shows on the CPU that a
network replaced by its cell-mean constant rates, or fed a wrong group table, fails it.
"""

import numpy as np

from oracle import collision as col
from oracle import lattice as L
from oracle import stepper as S

_PERM, _SIGN = L.moment_action_tables()   # (P_g m)_k = sign[g, k] m[perm[g, k]]


def bf16(x):
    """Round to BF16 (nearest even) through FP32, as the kernels round FP32 values."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint32) << 16
    return r.view(np.float32).astype(np.float64)


def ulp_bf16(v):
    """Spacing of BF16 numbers at |v| (8 significant bits)."""
    v = np.abs(np.asarray(v, dtype=np.float64))
    return 2.0 ** (np.floor(np.log2(np.where(v > 0, v, 2.0 ** -126))) - 7)


def rates(f, theta, sizes=col.LAYER_SIZES):
    """Learned rates of the oracle with BF16 operands (the reference of the BF16 form)."""
    return col.nco_rates(f, theta, sizes, operand_round=bf16)


def rates_from_moments(m, theta, sizes=col.LAYER_SIZES, table=None, operand_round=bf16):
    """Rates with the group acting on moment vectors m (cells, 27) through a (perm, sign)
    table; with the true table this equals rates() up to FP64 rounding. Used to plant a
    wrong table or a moved input."""
    perm, sign = (_PERM, _SIGN) if table is None else table
    layers = col.unpack_theta(theta, sizes)
    acc = 0.0
    for g in range(L.G):
        acc = acc + col.phi_network(sign[g] * m[:, perm[g]], layers, operand_round)
    return 1.0 / col.tau_from_network(acc / L.G)


def rates_with_table(f, theta, sizes=col.LAYER_SIZES, table=None, operand_round=bf16):
    """rates_from_moments of the moments of populations f (..., 27)."""
    m = col.moments(np.asarray(f, dtype=np.float64).reshape(-1, 27))
    out = rates_from_moments(m, theta, sizes, table, operand_round)
    return out.reshape(np.shape(f)[:-1] + (sizes[-1],))


def tau_tilde_bound(f, theta, sizes=col.LAYER_SIZES, chunk=4096):
    """Per cell and output: the bound on |tau~_kernel - tau~_reference| (module docstring)."""
    layers = col.unpack_theta(theta, sizes)
    hidden = [(bf16(W), bf16(b)) for W, b in layers[:-1]]
    W_out = layers[-1][0]
    flat = np.asarray(f, dtype=np.float64).reshape(-1, 27)
    nout = sizes[-1]
    out = np.empty((flat.shape[0], nout))
    for a in range(0, flat.shape[0], chunk):
        m = col.moments(flat[a: a + chunk])
        mb = bf16(m)
        n = m.shape[0]
        jac = np.zeros((n, nout, 27))     # d tau~ / d m (sum over g; divided by 48 below)
        hflip = np.zeros((n, nout))
        accum = np.zeros((n, nout))
        for g in range(L.G):
            h = _SIGN[g] * mb[:, _PERM[g]]
            acts, masks = [h], []
            for W, b in hidden:
                z = h @ W.T + b
                masks.append(z > 0.0)
                h = np.maximum(z, 0.0)
                acts.append(h)
                h = bf16(h)
            accum += np.abs(acts[-1]) @ np.abs(W_out).T
            grad = W_out[None, :, :] * masks[-1][:, None, :]     # d tau~ / d z of the last hidden layer
            for li in range(len(hidden) - 1, -1, -1):
                d_in = grad @ hidden[li][0]                         # d tau~ / d (input of layer li)
                if li > 0:
                    h_in = bf16(acts[li])                           # the rounded activation layer li reads
                    hflip = np.maximum(hflip, (np.abs(d_in) * ulp_bf16(h_in)[:, None, :]).max(axis=2))
                    grad = d_in * masks[li - 1][:, None, :]
                else:
                    jac[:, :, _PERM[g]] += d_in * _SIGN[g][None, None, :]
        jac /= L.G
        terms = np.sort(np.abs(jac) * ulp_bf16(m)[:, None, :], axis=2)
        first = terms[:, :, -1] + terms[:, :, -2]
        out[a: a + chunk] = 2.0 * (first + 4.0 * hflip / L.G + 1e-6 + 1e-5 * accum / L.G)
    return out.reshape(np.shape(f)[:-1] + (nout,))


def rate_bound(f, theta, sizes=col.LAYER_SIZES):
    """Bound on |omega_kernel - omega_reference| per cell and order group."""
    return 0.5 * tau_tilde_bound(f, theta, sizes)


def population_bound(f, rate_tol):
    """|d f*_i| <= sum_n rate_tol_n |(M^-1 m_(order n+3))_i| per cell and population."""
    m = col.moments(np.asarray(f, dtype=np.float64))
    out = np.zeros(np.shape(f))
    for n in range(4):
        mn = np.where(L.MOMENT_ORDER == n + 3, m, 0.0)
        out += rate_tol[..., n: n + 1] * np.abs(mn @ L.M_INV.T)
    return out


def storage_round(dev, storage):
    """The storage format's rounding of a deviation f - w (FP32 storage: none)."""
    if storage == "f16":
        return np.asarray(dev, dtype=np.float64).astype(np.float16).astype(np.float64)
    if storage == "bf16":
        return bf16(dev)
    return np.asarray(dev, dtype=np.float64)


def stream(fstar, bc):
    if bc == "periodic":
        return S.stream_periodic(fstar)
    if bc == "mirror":
        return S.stream_mirror(fstar)
    if bc == "tgv_reduced":
        return S.stream_tgv_reduced(fstar)
    raise ValueError(bc)


def step_reference(start, tau, theta, sizes=col.LAYER_SIZES, bc="periodic", rate_fn=None):
    """One NCO step of the BF16-operand oracle from populations (nz, ny, nx, 27), with the
    bound on each post-streaming population. rate_fn(f) replaces the reference rates
    (to plant a mistake); the bound is always the reference's."""
    f = np.asarray(start, dtype=np.float64)
    w = rates(f, theta, sizes) if rate_fn is None else rate_fn(f)
    post = col.mrt_collide(f, tau, w)
    bound = population_bound(f, rate_bound(f, theta, sizes))
    return stream(post, bc), stream(bound, bc)


def within(got, ref, bound, storage):
    """Boolean array: is every stored value a storage rounding of a value within the bound
    (plus 1e-5 max|ref| for FP32 arithmetic) of the reference?"""
    slack = bound + 1e-5 * np.abs(ref).max()
    lo = storage_round(ref - L.W - slack, storage) + L.W
    hi = storage_round(ref - L.W + slack, storage) + L.W
    # the FP32 store of an FP32 deviation and the FP32 sum w + (f - w) of a state read-back
    # are two more roundings
    eps = 2.0 ** -22 * (np.abs(ref) + L.W)
    got = np.asarray(got, dtype=np.float64)
    return (got >= lo - eps) & (got <= hi + eps)


def sensitive_theta(theta, sizes=col.LAYER_SIZES, scale=30.0):
    """Weights whose rates depend strongly on the state: the first layer's weights scaled
    (seed-0 Kaiming weights give rates that vary by < 0.01 across random cells; x30 makes
    them span about 1.15..1.84). Biases and other layers unchanged; FP32-representable."""
    th = np.asarray(theta, dtype=np.float32).copy()
    th[: sizes[0] * sizes[1]] *= np.float32(scale)
    return th


DEEP_SIZES = (27, 20, 20, 20, 4)

# Inputs of the GPU parity tests of the BF16 network, shared with the CPU test that shows
# the tolerance rejects planted mistakes on exactly these inputs:
# name: (shape (nz, ny, nx), population seed, nu, layer sizes, boundaries)
CASES = {
    "ragged": ((7, 6, 5), 17, 0.02, col.LAYER_SIZES, ("periodic", "mirror")),   # 210 = 128 + 82 cells
    "large_ragged": ((9, 17, 33), 19, 0.01, col.LAYER_SIZES, ("periodic",)),   # 5049 cells, 40 tiles
    "deep": ((7, 6, 5), 43, 0.02, DEEP_SIZES, ("periodic",)),
}


def case_theta(sizes, weights):
    """'seed0': the Kaiming-uniform draws of seed 0; 'sensitive': the same with W1 x 30."""
    import lbm_inputs
    th = lbm_inputs.nco_parameters(0, sizes).astype(np.float32)
    return th if weights == "seed0" else sensitive_theta(th, sizes)


def stored_start(f0_soa, storage):
    """The pre-collision populations (nz, ny, nx, 27) a context holds after lbm_set_state
    of f0 (27, nz, ny, nx): w + (f0 - w) rounded to the storage format, summed in FP32."""
    f = np.moveaxis(np.asarray(f0_soa, dtype=np.float64), 0, -1)
    dev = storage_round(f.astype(np.float32).astype(np.float64) - L.W, storage)
    return (dev.astype(np.float32) + L.W.astype(np.float32)).astype(np.float64)
