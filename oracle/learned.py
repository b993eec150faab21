"""Oracle of the learned preconditioner: grid transfer and a small 3D convolutional U-Net.

TEST INFRASTRUCTURE ONLY (see the package header).

Not in the paper: the learned coarse correction for the pressure-Poisson solve (a16 of the build's
scope) restricts the nodal residual to a uniform grid of D^3 cells (D = 64 on the workloads),
adds a second channel log(1/rho~) there, applies a convolutional network and prolongates its
output back to the nodes; flexible CG uses z = c(r) + omega D^-1 (r - A c(r)), omega = 2/3.

* Grid transfer. P_g (nodes x cells) interpolates cell-centred values trilinearly to the node
  positions (constant extrapolation beyond the outermost cell centres). The residual channel is
  R r / s(r) with R = P_g^T (the adjoint: residuals are integrals against test functions) and
  s(r) = sqrt(r.r / D^3); the density channel is the P_g-weighted mean (P_g^T f) / (P_g^T 1) of
  f = log(1/rho(clamp(phi~))). The correction is c(r) = s(r) out_scale P_g net(x(r)).
* Network (4 levels, C channels, C = 16): enc0 = relu(conv3(x)) at D; enc_l = relu(conv3(pool(
  enc_{l-1}))) at D/2^l for l = 1..3; dec_l = relu(conv3(up(dec_{l+1}) + enc_l)) for l = 2..0 with
  dec_3 = enc_3; out = conv1(dec_0) (linear, one channel). conv3: 3x3x3, zero padding, bias;
  pool: 2x2x2 mean; up: nearest-neighbour copy. Activations are (C, D, D, D) arrays. forward and
  backward take optional rounding functions (bf16_round) applied where a bfloat16 implementation
  stores a tensor: every activation, and every gradient after a ReLU mask.
* Training pairs of a mean-free error sample e: input x(A e); loss = the relative energy norm
  (e - c)^T A (e - c) / e^T A e of the error the correction leaves; Adam. The grid target
  cell_mean(e) / s(A e) only sets the default output scale (its RMS).

Pins (tests/test_oracle_learned.py): hand backward = central finite differences; a delta
kernel reproduces its input; pool/up adjointness; P_g partition of unity and exact interpolation
of trilinear-in-cell-centre fields; R = P_g^T; bf16_round = the library's bfloat16 conversion
(ties to even); a constant network gives the closed-form correction s out_scale c; the
correction is positively homogeneous and zero for r = 0, and a zero network leaves Jacobi;
constant errors give zero targets (null space); the energy-loss gradient = central finite
differences of the energy loss, and a zero network gives loss 1; flexible CG with a fixed
preconditioner equals Jacobi-PCG. The network's values are otherwise only defined by this code: parity unpinned beyond
these checks.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

MAXD = 20


# ------------------------------------------------------------------ grid transfer
def grid_prolongation(node_int: np.ndarray, extent, D: int) -> sp.csr_matrix:
    """P_g (n_nodes x D^3): trilinear interpolation of cell-centred values at the nodes.
    Cell c = (i, j, k) (x fastest, index i + D (j + D k)) has centre ((i + 0.5)/D) * L."""
    x = np.asarray(node_int, dtype=np.float64) / float(1 << MAXD)        # unit-cube coordinates
    s = x * D - 0.5
    i0 = np.clip(np.floor(s).astype(np.int64), 0, D - 2)
    t = np.clip(s - i0, 0.0, 1.0)
    rows, cols, vals = [], [], []
    n = len(x)
    for c in range(8):
        b = [(c >> d) & 1 for d in range(3)]
        w = np.ones(n)
        idx = np.zeros(n, dtype=np.int64)
        mul = 1
        for d in range(3):
            w = w * (t[:, d] if b[d] else 1.0 - t[:, d])
            idx = idx + (i0[:, d] + b[d]) * mul
            mul *= D
        rows.append(np.arange(n))
        cols.append(idx)
        vals.append(w)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, D ** 3))


def cell_mean(Pg: sp.csr_matrix, f: np.ndarray, D: int) -> np.ndarray:
    """P_g-weighted mean (P_g^T f) / (P_g^T 1) per cell, 0 in cells no node reaches; (D, D, D)."""
    wsum = Pg.T @ np.ones(Pg.shape[0])
    num = Pg.T @ f
    out = np.zeros_like(num)
    nz = wsum > 0
    out[nz] = num[nz] / wsum[nz]
    return out.reshape(D, D, D)


def log_inv_rho(co, phi_t: np.ndarray) -> np.ndarray:
    """log(1/rho(phi*)) at the nodes, phi* = clamp(phi~, -1, 1) (co: oracle.fem.Coeffs)."""
    return -np.log(co.rho(phi_t))


def input_scale(r: np.ndarray, D: int) -> float:
    """s(r) = sqrt(r.r / D^3): the residual channel is fed as R r / s and the network's output is
    scaled back by s, which makes the correction positively homogeneous in r."""
    return float(np.sqrt(np.dot(r, r) / D ** 3))


def restrict_inputs(Pg: sp.csr_matrix, r: np.ndarray, lr_cell: np.ndarray, D: int):
    """The two input channels (2, D, D, D): R r / s(r) and the cell mean of log(1/rho); and s."""
    s = input_scale(r, D)
    rr = (Pg.T @ r).reshape(D, D, D)
    return np.stack([rr / s if s > 0 else 0.0 * rr, lr_cell]), s


def training_target(Pg: sp.csr_matrix, e: np.ndarray, s: float, D: int) -> np.ndarray:
    """Grid target of an error sample e (residual r = A e): the cell mean of the mean-free e
    (constants are the pure-Neumann operator's null space) divided by s(r)."""
    return cell_mean(Pg, e - np.mean(e), D) / s


def coarse_correction(P, Pg, r, lr_cell, D, out_scale, round_act=None):
    """c(r) = s(r) out_scale P_g net(R r / s(r), lr); zero for r = 0."""
    x, s = restrict_inputs(Pg, r, lr_cell, D)
    if s == 0.0:
        return np.zeros(Pg.shape[0])
    out, _ = forward(P, x, round_act)
    return s * out_scale * (Pg @ out.ravel())


def precondition(P, Pg, A, r, lr_cell, D, out_scale, dinv, omega=2.0 / 3.0, round_act=None):
    """Two-level preconditioner used inside flexible CG: the learned coarse correction c(r), then
    one damped Jacobi step on the residual it leaves, z = c + omega D^-1 (r - A c)."""
    c = coarse_correction(P, Pg, r, lr_cell, D, out_scale, round_act)
    return c + omega * dinv * (r - A @ c)


# ------------------------------------------------------------------ layers (arrays: (C, D, D, D) with index [c, z, y, x])
TAPS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shift(a, dx, dy, dz):
    """s[c, z, y, x] = a[c, z+dz, y+dy, x+dx] with zeros outside."""
    p = np.pad(a, ((0, 0), (1, 1), (1, 1), (1, 1)))
    D = a.shape[1]
    return p[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + D, 1 + dx:1 + dx + D]


def conv3(x, W, b):
    """W (27, Cout, Cin) indexed by tap t = TAPS index; y[co] = sum_t sum_ci W[t,co,ci] x_shift_t[ci] + b."""
    y = np.zeros((W.shape[1],) + x.shape[1:])
    for t, (dx, dy, dz) in enumerate(TAPS):
        y += np.tensordot(W[t], _shift(x, dx, dy, dz), axes=([1], [0]))
    return y + b[:, None, None, None]


def conv3_backward(x, W, gy):
    gW = np.zeros_like(W)
    gx = np.zeros_like(x)
    for t, (dx, dy, dz) in enumerate(TAPS):
        xs = _shift(x, dx, dy, dz)
        gW[t] = np.tensordot(gy, xs, axes=([1, 2, 3], [1, 2, 3]))
        gx += _shift(np.tensordot(W[t], gy, axes=([0], [0])), -dx, -dy, -dz)
    return gx, gW, gy.sum(axis=(1, 2, 3))


def pool(x):
    C, D = x.shape[0], x.shape[1]
    return x.reshape(C, D // 2, 2, D // 2, 2, D // 2, 2).mean(axis=(2, 4, 6))


def pool_backward(gy):
    return np.repeat(np.repeat(np.repeat(gy, 2, 1), 2, 2), 2, 3) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 1), 2, 2), 2, 3)


def up_backward(gy):
    C, D = gy.shape[0], gy.shape[1]
    return gy.reshape(C, D // 2, 2, D // 2, 2, D // 2, 2).sum(axis=(2, 4, 6))


# ------------------------------------------------------------------ network
LAYERS = ["enc0", "enc1", "enc2", "enc3", "dec2", "dec1", "dec0"]


def init_params(C: int = 16, cin: int = 2, seed: int = 0):
    """He-normal conv weights (seeded), zero biases. Returns a dict of arrays."""
    rng = np.random.default_rng(seed)
    P = {}
    for name in LAYERS:
        ci = cin if name == "enc0" else C
        P[name + ".W"] = rng.standard_normal((27, C, ci)) * np.sqrt(2.0 / (27 * ci))
        P[name + ".b"] = np.zeros(C)
    P["out.W"] = rng.standard_normal((1, C)) * np.sqrt(1.0 / C)
    P["out.b"] = np.zeros(1)
    return P


def forward(P, x, round_act=None):
    """Forward pass; round_act (optional) rounds each stored activation (e.g. to bfloat16) the way
    a reduced-precision implementation stores them. Returns (out (D,D,D), cache)."""
    rnd = round_act or (lambda a: a)
    cache = {"x": rnd(x)}
    a = cache["x"]
    enc = []
    for l in range(4):
        inp = a if l == 0 else rnd(pool(a))
        z = conv3(inp, P[f"enc{l}.W"], P[f"enc{l}.b"])
        a = rnd(np.maximum(z, 0.0))
        cache[f"enc{l}.in"] = inp
        cache[f"enc{l}.out"] = a
        enc.append(a)
    d = enc[3]
    for l in (2, 1, 0):
        inp = rnd(up(d) + enc[l])
        z = conv3(inp, P[f"dec{l}.W"], P[f"dec{l}.b"])
        d = rnd(np.maximum(z, 0.0))
        cache[f"dec{l}.in"] = inp
        cache[f"dec{l}.out"] = d
    out = np.tensordot(P["out.W"], d, axes=([1], [0]))[0] + P["out.b"][0]
    return out, cache


def backward(P, cache, gout, round_grad=None):
    """Gradients of all parameters given dL/d(out) (D,D,D). round_grad (optional) rounds the
    gradient at each conv output after the ReLU mask, where a reduced-precision implementation
    stores it as the operand of its transposed convolution and weight-gradient contraction."""
    rg = round_grad or (lambda a: a)
    G = {}
    d0 = cache["dec0.out"]
    G["out.W"] = np.tensordot(gout[None], d0, axes=([1, 2, 3], [1, 2, 3]))
    G["out.b"] = np.array([gout.sum()])
    gd = P["out.W"][0][:, None, None, None] * gout[None]
    genc = {l: np.zeros_like(cache[f"enc{l}.out"]) for l in range(4)}
    for l in (0, 1, 2):
        gz = rg(gd * (cache[f"dec{l}.out"] > 0))
        gin, G[f"dec{l}.W"], G[f"dec{l}.b"] = conv3_backward(cache[f"dec{l}.in"], P[f"dec{l}.W"], gz)
        genc[l] += gin                      # skip connection
        gd = up_backward(gin)               # to dec_{l+1} (= enc3 for l = 2)
    genc[3] += gd
    ga = None
    for l in (3, 2, 1, 0):
        g = genc[l] + (ga if ga is not None else 0.0)
        gz = rg(g * (cache[f"enc{l}.out"] > 0))
        gin, G[f"enc{l}.W"], G[f"enc{l}.b"] = conv3_backward(cache[f"enc{l}.in"], P[f"enc{l}.W"], gz)
        ga = pool_backward(gin) if l > 0 else None
    return G


def energy_loss_and_grad(P, Pg, A, e, x, s, D, out_scale, round_act=None):
    """Training loss of one pair: the relative energy norm of the error the correction leaves,
    c = s out_scale P_g out(x), d = e - c, loss = d^T A d / e^T A e (e mean-free, A symmetric),
    and dL/d(out) = -2 s out_scale P_g^T A d / e^T A e. Returns (loss, gout (D,D,D), cache)."""
    out, cache = forward(P, x, round_act)
    c = s * out_scale * (Pg @ out.ravel())
    d = e - c
    Ad = A @ d
    eae = float(e @ (A @ e))
    loss = float(d @ Ad) / eae
    gout = (-2.0 * s * out_scale / eae) * (Pg.T @ Ad)
    return loss, gout.reshape(D, D, D), cache


def flatten(P) -> np.ndarray:
    """Parameters (or gradients) as one vector: per layer of LAYERS its W then b, then out.W, out.b."""
    keys = [k for name in LAYERS for k in (name + ".W", name + ".b")] + ["out.W", "out.b"]
    return np.concatenate([np.asarray(P[k], dtype=np.float64).ravel() for k in keys])


def unflatten(v: np.ndarray, C: int = 16, cin: int = 2):
    P, o = {}, 0
    shapes = []
    for name in LAYERS:
        ci = cin if name == "enc0" else C
        shapes += [(name + ".W", (27, C, ci)), (name + ".b", (C,))]
    shapes += [("out.W", (1, C)), ("out.b", (1,))]
    for k, shp in shapes:
        n = int(np.prod(shp))
        P[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(shp).copy()
        o += n
    assert o == len(v)
    return P


def bf16_round(a) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def loss_and_grad(out, target):
    diff = out - target
    return 0.5 * float(np.mean(diff ** 2)), diff / diff.size


class Adam:
    def __init__(self, P, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps, self.t = lr, b1, b2, eps, 0
        self.m = {k: np.zeros_like(v) for k, v in P.items()}
        self.v = {k: np.zeros_like(v) for k, v in P.items()}

    def step(self, P, G):
        self.t += 1
        for k in P:
            self.m[k] = self.b1 * self.m[k] + (1 - self.b1) * G[k]
            self.v[k] = self.b2 * self.v[k] + (1 - self.b2) * G[k] ** 2
            mh = self.m[k] / (1 - self.b1 ** self.t)
            vh = self.v[k] / (1 - self.b2 ** self.t)
            P[k] = P[k] - self.lr * mh / (np.sqrt(vh) + self.eps)


def fcg(A, b, precond, x0=None, rtol=1e-8, maxit=10000, mean_zero=False):
    """Flexible CG (Polak-Ribiere beta) for a variable preconditioner z = precond(r)."""
    b = np.asarray(b, dtype=np.float64).copy()
    if mean_zero:
        b -= b.mean()
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    bn = np.linalg.norm(b)
    z = precond(r)
    p = z.copy()
    rz = r @ z
    it = 0
    while np.linalg.norm(r) > rtol * bn and it < maxit:
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r_new = r - alpha * q
        z_new = precond(r_new)
        beta = (z_new @ (r_new - r)) / rz
        rz = r_new @ z_new
        p = z_new + beta * p
        r = r_new
        it += 1
    if mean_zero:
        x -= x.mean()
    return x, it, np.linalg.norm(r) / bn
