"""Oracle for the learned gauge-covariant preconditioner network -- test infrastructure only.

The paper closes (Sec. 4) by naming the search for a better preconditioner than j-step Jacobi as
future work.  The network below is such a preconditioner: it is linear in the spinor, so M_net is
a fixed linear operator that block BiCGGR can use, and it is gauge covariant, so it commutes with
gauge transformations as A does.

Layer (maps C_in channels to C_out channels of spinor fields psi_c(x), spin x colour):
    out_{c'}(x) = sum_{d=0..8} sum_c W[d, c', c] (T_d psi_c)(x)
    T_0 psi = psi,
    T_{1+mu} psi (x) = U_mu(x) psi(x + mu),      T_{5+mu} psi (x) = U_mu(x - mu)^H psi(x - mu),
with W[d, c', c] a complex 4x4 matrix acting on spin (colour is moved only by the links).
Network: layers with channels (1, C, ..., C, 1) applied in order, no non-linearity.
Loss over a batch of pairs (r_i, e_i = A^{-1} r_i), the L columns of R and E:
    loss = (1/L) sum_i ||N(r_i) - e_i||^2 / ||e_i||^2.
Gradient: G = d loss / d conj(W) (Wirtinger), by reverse-mode differentiation through the
adjoint layers; the real gradient with respect to (Re W, Im W) is (2 Re G, 2 Im G).
Training step: Adam on the real parameters (Re W, Im W).

Parity status: pinned (tests/test_oracle_network.py: finite differences of the loss, linearity,
gauge covariance, the one-layer Wilson hopping special case, Adam's closed-form first step).
Layouts: activations [C][V][4 spin][3 colour][L]; weights per layer [9][C_out][C_in][4][4].
"""
from __future__ import annotations

import numpy as np

NDIR = 9


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def transport(U, lat, psi, d):
    """T_d psi for psi [V][4][3][L]."""
    if d == 0:
        return psi
    if d <= 4:
        mu = d - 1
        return np.einsum("vab,vsbl->vsal", U[:, mu], psi[lat.fwd[mu]])
    mu = d - 5
    return np.einsum("vab,vsbl->vsal", _dag(U[lat.bwd[mu], mu]), psi[lat.bwd[mu]])


def transport_adjoint(U, lat, phi, d):
    """T_d^H phi: T_0^H = 1, T_{1+mu}^H = T_{5+mu}, T_{5+mu}^H = T_{1+mu}."""
    if d == 0:
        return phi
    return transport(U, lat, phi, d + 4 if d <= 4 else d - 4)


def layer(U, lat, W, x):
    """out[c'] = sum_d sum_c W[d, c', c] T_d x[c];  x [C_in][V][4][3][L]."""
    cin = x.shape[0]
    cout = W.shape[1]
    out = np.zeros((cout,) + x.shape[1:], dtype=complex)
    for d in range(NDIR):
        for c in range(cin):
            t = transport(U, lat, x[c], d)
            for co in range(cout):
                out[co] += np.einsum("st,vtal->vsal", W[d, co, c], t)
    return out


def forward(U, lat, weights, r):
    """N(r) and the layer inputs a_0 .. a_{n-1} (kept for the gradient)."""
    acts = [r[None]]
    for W in weights:
        acts.append(layer(U, lat, W, acts[-1]))
    return acts[-1][0], acts[:-1]


def loss_and_grad(U, lat, weights, R, E):
    """loss = (1/L) sum_i ||N(r_i) - e_i||^2 / ||e_i||^2 and G_l = d loss / d conj(W_l)."""
    L = R.shape[-1]
    Y, acts = forward(U, lat, weights, R)
    en2 = np.sum(np.abs(E.reshape(-1, L)) ** 2, axis=0)
    diff = Y - E
    loss = float(np.mean(np.sum(np.abs(diff.reshape(-1, L)) ** 2, axis=0) / en2))
    delta = (diff / (L * en2))[None]                       # d loss / d conj(Y)
    grads = [None] * len(weights)
    for li in range(len(weights) - 1, -1, -1):
        W, a = weights[li], acts[li]
        cout, cin = W.shape[1], W.shape[2]
        G = np.zeros_like(W)
        prev = np.zeros_like(a)
        for d in range(NDIR):
            for c in range(cin):
                t = transport(U, lat, a[c], d)
                for co in range(cout):
                    G[d, co, c] = np.einsum("vsal,vtal->st", delta[co], np.conj(t))
                    prev[c] += transport_adjoint(
                        U, lat, np.einsum("ts,vtal->vsal", np.conj(W[d, co, c]), delta[co]), d)
        grads[li] = G
        delta = prev
    return loss, grads


def adam_step(weights, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step on the real parameters (Re W, Im W) with real gradient (2 Re G, 2 Im G).
    ``state`` is a dict with 't' and per-layer first/second moments of the real parameters."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    new = []
    for li, (W, G) in enumerate(zip(weights, grads)):
        p = np.stack([W.real, W.imag])
        g = np.stack([2 * G.real, 2 * G.imag])
        m = state.setdefault(("m", li), np.zeros_like(p))
        v = state.setdefault(("v", li), np.zeros_like(p))
        m[...] = beta1 * m + (1 - beta1) * g
        v[...] = beta2 * v + (1 - beta2) * g * g
        mhat = m / (1 - beta1 ** t)
        vhat = v / (1 - beta2 ** t)
        p = p - lr * mhat / (np.sqrt(vhat) + eps)
        new.append(p[0] + 1j * p[1])
    return new
