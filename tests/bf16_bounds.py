"""Error bounds for the surrogate network evaluated as tensor cores take it:
the input of every matrix product rounded to bfloat16 (forward: f, h1, h2;
backward: dw, dz2, dz1), each to nearest with relative error <= u = 2^-9 (8
significant bits).  The weights are the same on both sides (already rounded).

Per link n, a first-order running-error bound c_n bounds, component by
component, how far that link's share of each result moves: every rounding
contributes u |x| at its tensor and travels through the following products
with the absolute values of their other factors, through tanh with its
derivative 1 - h^2 (and through 1 - h^2 in the backward pass with
|d(1 - h^2)| = 2 |h| |dh|).  The loss and the parameter gradients are sums
over the links, so two bounds follow:

  worst case      sum_n c_n                       (rigorous, first order)
  probabilistic   sqrt(sum_n c_n^2)               (rounding errors of different
                                                   links independent, zero mean)

The links' errors cancel in the sums as independent rounding errors do
(Higham and Mary, SIAM J. Sci. Comput. 41 (2019) A2815), so a result more
than lambda = 3 probabilistic bounds away from the exact one has a
probability below 2 exp(-3 lambda^2 / 2) ~ 3e-6 per component for errors
uniform within +-c_n (variance c_n^2 / 3).  The force of one link is not a
sum over links: its bound is c_n itself.

A separate term covers fp32 arithmetic on the device (features, generators
and the sums over links accumulated in fp32): (n_links + 64) 2^-24 times the
absolute-value product, added to both bounds.

Test infrastructure: pure error analysis; it shares no code with the library
or the oracle."""
import numpy as np

U_BF16 = 2.0 ** -9
U_F32 = 2.0 ** -24
LAMBDA = 3.0


def network_bounds(p, f, G, F):
    """Exact results and their bounds for the loss, every parameter gradient
    and the surrogate force F^ of the 24-32-32-24 tanh network with weights
    p, features f [..., 24], generators G [..., 24, 8] and target F [..., 8].

    Returns (exact, worst, prob): dicts with "loss", "W1" .. "b3" and
    "force" (the force's two bounds are the same)."""
    u, A = U_BF16, np.abs
    fl = f.reshape(-1, 24)
    Gf = G.reshape(-1, 24, 8)
    Ff = F.reshape(-1, 8)
    n = fl.shape[0]
    W1, W2, W3 = p["W1"], p["W2"], p["W3"]
    # exact network
    h1 = np.tanh(fl @ W1.T + p["b1"])
    h2 = np.tanh(h1 @ W2.T + p["b2"])
    w = h2 @ W3.T + p["b3"]
    force = np.einsum("nk,nka->na", w, Gf)
    e = force - Ff
    dw = 2.0 * np.einsum("na,nka->nk", e, Gf) / n
    g3 = dw @ W3
    dz2 = g3 * (1 - h2 ** 2)
    g2 = dz2 @ W2
    dz1 = g2 * (1 - h1 ** 2)
    exact = {"loss": float(np.sum(e * e) / n), "W3": dw.T @ h2, "b3": dw.sum(0), "W2": dz2.T @ h1,
             "b2": dz2.sum(0), "W1": dz1.T @ fl, "b1": dz1.sum(0), "force": force.reshape(F.shape)}
    # forward roundings, per link
    d_f = u * A(fl)
    d_h1 = (1 - h1 ** 2) * (d_f @ A(W1).T)
    d_h1q = d_h1 + u * A(h1)
    d_h2 = (1 - h2 ** 2) * (d_h1q @ A(W2).T)
    d_h2q = d_h2 + u * A(h2)
    d_w = d_h2q @ A(W3).T
    d_e = np.einsum("nk,nka->na", d_w, A(Gf))
    # backward roundings, per link
    d_dw = 2.0 * np.einsum("na,nka->nk", d_e, A(Gf)) / n
    d_dwq = d_dw + u * A(dw)
    d_dz2 = (d_dwq @ A(W3)) * (1 - h2 ** 2) + A(g3) * 2 * A(h2) * d_h2
    d_dz2q = d_dz2 + u * A(dz2)
    d_dz1 = (d_dz2q @ A(W2)) * (1 - h1 ** 2) + A(g2) * 2 * A(h1) * d_h1
    d_dz1q = d_dz1 + u * A(dz1)
    # per-link contributions c_n (leading axis n) and the fp32 terms
    per_link = {
        "loss": 2.0 * np.sum(A(e) * d_e, axis=1) / n,
        "W3": d_dwq[:, :, None] * A(h2)[:, None, :] + A(dw)[:, :, None] * d_h2q[:, None, :],
        "b3": d_dwq,
        "W2": d_dz2q[:, :, None] * A(h1)[:, None, :] + A(dz2)[:, :, None] * d_h1q[:, None, :],
        "b2": d_dz2q,
        "W1": d_dz1q[:, :, None] * A(fl)[:, None, :] + A(dz1)[:, :, None] * d_f[:, None, :],
        "b1": d_dz1q,
    }
    acc = (n + 64) * U_F32
    fp32 = {"loss": acc * float(np.sum(e * e)) / n, "W3": acc * (A(dw).T @ A(h2)), "b3": acc * A(dw).sum(0),
            "W2": acc * (A(dz2).T @ A(h1)), "b2": acc * A(dz2).sum(0), "W1": acc * (A(dz1).T @ A(fl)),
            "b1": acc * A(dz1).sum(0)}
    worst = {k: v.sum(0) + fp32[k] for k, v in per_link.items()}
    prob = {k: np.sqrt((v * v).sum(0)) + fp32[k] for k, v in per_link.items()}
    fb = (np.einsum("nk,nka->na", d_w, A(Gf)) + 64 * U_F32 * np.einsum("nk,nka->na", A(w), A(Gf))).reshape(F.shape)
    worst["force"] = prob["force"] = fb
    return exact, worst, prob


def ratio(got, exact, bound):
    """Largest |got - exact| / bound over the components."""
    got, exact, bound = (np.asarray(a, dtype=np.float64) for a in (got, exact, bound))
    return float(np.max(np.abs(got - exact) / (bound + 1e-300)))
