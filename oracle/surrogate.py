"""Learned fermion-force surrogate (a workload of the build, not of the paper):
loop features, staple generators, the MLP and its hand-written backward pass,
in float64.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Per link (x, mu) and each of the three nu != mu (in increasing order), eight
staples S close a loop U_mu(x) S:
  0 plaquette up     U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
  1 plaquette down   U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)
  2 rect 2mu x nu up, link first    U_mu(x+mu) U_nu(x+2mu) U_mu(x+mu+nu)^+ U_mu(x+nu)^+ U_nu(x)^+
  3 rect 2mu x nu up, link second   U_nu(x+mu) U_mu(x+nu)^+ U_mu(x-mu+nu)^+ U_nu(x-mu)^+ U_mu(x-mu)
  4 rect 2mu x nu down, link first  U_mu(x+mu) U_nu(x+2mu-nu)^+ U_mu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)
  5 rect 2mu x nu down, link second U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_mu(x-mu-nu)^+ U_nu(x-mu-nu) U_mu(x-mu)
  6 rect mu x 2nu up     U_nu(x+mu) U_nu(x+mu+nu) U_mu(x+2nu)^+ U_nu(x+nu)^+ U_nu(x)^+
  7 rect mu x 2nu down   U_nu(x+mu-nu)^+ U_nu(x+mu-2nu)^+ U_mu(x-2nu)^+ U_nu(x-2nu) U_nu(x-nu)
so staple k = 8 * (index of nu among the three) + j.
  features  f_k = Re tr(U_mu(x) S_k) / 3              (gauge invariant)
  generators G_{k,a} = Re tr(i T_a U_mu(x) S_k)        (force of each loop)
  MLP       h1 = tanh(W1 f + b1), h2 = tanh(W2 h1 + b2), w = W3 h2 + b3   (24-32-32-24);
            on tensor cores f, h1, h2 enter the products rounded to bfloat16 (quant=True)
  surrogate F^_a = sum_k w_k G_{k,a}                  (gauge covariant)
  loss      mean over links of sum_a (F^_a - F_a)^2
"""
import numpy as np

from . import lattice as lat
from .su3 import T, dag

SIZES = (24, 32, 32, 24)


def _mm(*ms):
    out = ms[0]
    for m in ms[1:]:
        out = np.einsum("...ij,...jk->...ik", out, m)
    return out


def _at(u, nu, shifts):
    """U_nu at x + sum(sign * dir) for shifts = [(dir, sign), ...]."""
    v = u[nu]
    for d, sg in shifts:
        v = lat.shift_fwd(v, d) if sg > 0 else lat.shift_bwd(v, d)
    return v


def staples(u, mu):
    """The 24 staples of every link in direction mu: [t, z, y, x, 24, 3, 3]."""
    out = []
    for nu in [n for n in range(4) if n != mu]:
        U = lambda d, sh: _at(u, d, sh)            # noqa: E731
        m, n = mu, nu
        out += [
            _mm(U(n, [(m, 1)]), dag(U(m, [(n, 1)])), dag(U(n, []))),
            _mm(dag(U(n, [(m, 1), (n, -1)])), dag(U(m, [(n, -1)])), U(n, [(n, -1)])),
            _mm(U(m, [(m, 1)]), U(n, [(m, 1), (m, 1)]), dag(U(m, [(m, 1), (n, 1)])), dag(U(m, [(n, 1)])),
                dag(U(n, []))),
            _mm(U(n, [(m, 1)]), dag(U(m, [(n, 1)])), dag(U(m, [(m, -1), (n, 1)])), dag(U(n, [(m, -1)])),
                U(m, [(m, -1)])),
            _mm(U(m, [(m, 1)]), dag(U(n, [(m, 1), (m, 1), (n, -1)])), dag(U(m, [(m, 1), (n, -1)])),
                dag(U(m, [(n, -1)])), U(n, [(n, -1)])),
            _mm(dag(U(n, [(m, 1), (n, -1)])), dag(U(m, [(n, -1)])), dag(U(m, [(m, -1), (n, -1)])),
                U(n, [(m, -1), (n, -1)]), U(m, [(m, -1)])),
            _mm(U(n, [(m, 1)]), U(n, [(m, 1), (n, 1)]), dag(U(m, [(n, 1), (n, 1)])), dag(U(n, [(n, 1)])),
                dag(U(n, []))),
            _mm(dag(U(n, [(m, 1), (n, -1)])), dag(U(n, [(m, 1), (n, -1), (n, -1)])), dag(U(m, [(n, -1), (n, -1)])),
                U(n, [(n, -1), (n, -1)]), U(n, [(n, -1)])),
        ]
    return np.stack(out, axis=-3)


def features_and_generators(u):
    """f [4, t, z, y, x, 24] and G [4, t, z, y, x, 24, 8]."""
    fs, gs = [], []
    for mu in range(4):
        us = np.einsum("...ij,...kjl->...kil", u[mu], staples(u, mu))      # U S_k
        fs.append(np.real(np.trace(us, axis1=-2, axis2=-1)) / 3.0)
        gs.append(np.real(1j * np.einsum("aij,...kji->...ka", T, us)))
    return np.stack(fs), np.stack(gs)


def init_params(seed, scale=0.3):
    g = np.random.default_rng(seed)
    p = {}
    for i in range(3):
        n_in, n_out = SIZES[i], SIZES[i + 1]
        p[f"W{i + 1}"] = g.standard_normal((n_out, n_in)) * scale / np.sqrt(n_in)
        p[f"b{i + 1}"] = g.standard_normal(n_out) * 0.1
    return p


def forward(p, f, quant=False):
    """f [..., 24] -> w [..., 24], with the cache of the backward pass.

    quant=True is the network as tensor cores evaluate it: the input of every
    matrix product (f, h1, h2) rounded to bfloat16 (the weights are given
    already rounded), products and biases in full precision."""
    q = bf16_round if quant else (lambda a: a)     # noqa: E731
    fq = q(f)
    z1 = fq @ p["W1"].T + p["b1"]
    h1 = np.tanh(z1)
    h1q = q(h1)
    z2 = h1q @ p["W2"].T + p["b2"]
    h2 = np.tanh(z2)
    h2q = q(h2)
    w = h2q @ p["W3"].T + p["b3"]
    return w, (fq, h1, h2, h1q, h2q)


def backward(p, cache, dw, quant=False):
    """Gradients of a scalar L given dL/dw [..., 24] (summed over the leading
    axes).  With a quantised forward pass the rounding counts as the identity
    (straight-through): weight gradients use the rounded inputs, the tanh
    derivatives the unrounded activations.  quant=True also rounds the
    backward products' inputs dw, dz2, dz1 to bfloat16, as tensor cores take
    them (the bias gradients are sums of the same rounded values)."""
    q = bf16_round if quant else (lambda a: a)     # noqa: E731
    f, h1, h2, h1q, h2q = cache
    flat = lambda a: a.reshape(-1, a.shape[-1])     # noqa: E731
    f, h1, h2, h1q, h2q, dw = flat(f), flat(h1), flat(h2), flat(h1q), flat(h2q), flat(dw)
    dwq = q(dw)
    g = {"W3": dwq.T @ h2q, "b3": dwq.sum(0)}
    dz2 = (dwq @ p["W3"]) * (1 - h2 ** 2)
    dz2q = q(dz2)
    g["W2"], g["b2"] = dz2q.T @ h1q, dz2q.sum(0)
    dz1 = (dz2q @ p["W2"]) * (1 - h1 ** 2)
    dz1q = q(dz1)
    g["W1"], g["b1"] = dz1q.T @ f, dz1q.sum(0)
    return g


def surrogate_force(p, f, G, quant=False):
    """F^_a = sum_k w_k G_{k,a}: [4, t, z, y, x, 8]."""
    w, _ = forward(p, f, quant)
    return np.einsum("...k,...ka->...a", w, G)


def loss_and_grad(p, f, G, F, quant=False):
    """Mean over links of sum_a (F^_a - F_a)^2 and its parameter gradients."""
    w, cache = forward(p, f, quant)
    e = np.einsum("...k,...ka->...a", w, G) - F
    n = e[..., 0].size
    loss = float(np.sum(e * e) / n)
    dw = 2.0 * np.einsum("...a,...ka->...k", e, G) / n
    return loss, backward(p, cache, dw, quant)


def bf16_round(x):
    """Round float64 values to bfloat16 (through float32, nearest even), as float64."""
    b = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)
