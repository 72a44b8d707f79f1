"""Learned collision correction, FP64 oracle.  TEST INFRASTRUCTURE ONLY.

Not in the paper: a small MLP corrects the post-collision f of a coarse run
towards a 2x finer one.  Definitions (the library implements the same):

  basis   Phi [Q, Q]: modified Gram-Schmidt, in the weighted inner product
          <a, b> = sum_i w_i a_i b_i, of the monomials xi^m in graded order
          (total degree, then decreasing power of xi_0, then of xi_1), keeping
          the first Q that are linearly independent on the velocity set.
  input   z_k = sum_i Phi_ki f^neq_i  (non-equilibrium moments of the
          streamed populations, f^neq = f - f^eq), x = s (.) z
  network h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), o = W3 h2 + b3
          (widths Q -> 64 -> 64 -> Q; the library stores W in BF16)
  output  delta f_i = w_i sigma (P o)_i, where P removes the components along
          c in {1, xi_a, |xi|^2} in the weighted inner product, so that
          sum_i delta f_i c(xi_i) = 0: mass, momentum and energy are conserved
          exactly (up to rounding)
  loss    L = (1/M) sum_samples sum_i w_i ((P (o - y))_i)^2 with the target
          y = (f_fine - f_plain) / (w sigma)
"""
import numpy as np

HIDDEN = 64


def graded_monomials(D, max_degree):
    out = []
    for deg in range(max_degree + 1):
        if D == 2:
            for a in range(deg, -1, -1):
                out.append((a, deg - a))
        else:
            for a in range(deg, -1, -1):
                for b in range(deg - a, -1, -1):
                    out.append((a, b, deg - a - b))
    return out


def moment_basis(xi, w):
    """Phi [Q, Q] with sum_i w_i Phi_ki Phi_li = delta_kl."""
    Q, D = xi.shape
    rows = []
    for m in graded_monomials(D, 12):
        v = np.prod(xi ** np.array(m), axis=1)
        n0 = np.sqrt((w * v * v).sum())
        for r in rows:
            v = v - (w * v * r).sum() * r
        n = np.sqrt((w * v * v).sum())
        if n > 1e-9 * max(n0, 1.0):
            rows.append(v / n)
        if len(rows) == Q:
            break
    return np.array(rows)


def conservation_basis(xi):
    """c_k(xi_i) for c in {1, xi_0, .., xi_{D-1}, |xi|^2}: [D+2, Q]."""
    Q, D = xi.shape
    return np.vstack([np.ones(Q), xi.T, (xi ** 2).sum(1)])


def projector(xi, w):
    """P [Q, Q]: weighted-orthogonal projection onto the complement of the
    conserved functions."""
    C = conservation_basis(xi)
    G = (C * w) @ C.T
    return np.eye(len(w)) - C.T @ np.linalg.solve(G, C * w)


class MLP:
    def __init__(self, W1, b1, W2, b2, W3, b3, s_in, sigma):
        self.W1, self.b1, self.W2, self.b2, self.W3, self.b3 = (np.asarray(a, dtype=np.float64)
                                                                for a in (W1, b1, W2, b2, W3, b3))
        self.s_in = np.asarray(s_in, dtype=np.float64)
        self.sigma = float(sigma)

    def forward(self, x):
        """x [M, Q] (scaled inputs) -> o [M, Q] and the hidden activations."""
        h1 = np.tanh(x @ self.W1.T + self.b1)
        h2 = np.tanh(h1 @ self.W2.T + self.b2)
        o = h2 @ self.W3.T + self.b3
        return o, (x, h1, h2)

    def loss_and_grads(self, x, y, P, w):
        """Loss and gradients w.r.t. (W1, b1, W2, b2, W3, b3) for targets y [M, Q]."""
        M = len(x)
        o, (x, h1, h2) = self.forward(x)
        r = (o - y) @ P.T
        loss = float((w * r * r).sum() / M)
        g = 2.0 / M * (r * w) @ P                     # dL/do
        dW3 = g.T @ h2
        db3 = g.sum(0)
        dh2 = (g @ self.W3) * (1.0 - h2 * h2)
        dW2 = dh2.T @ h1
        db2 = dh2.sum(0)
        dh1 = (dh2 @ self.W2) * (1.0 - h1 * h1)
        dW1 = dh1.T @ x
        db1 = dh1.sum(0)
        return loss, (dW1, db1, dW2, db2, dW3, db3)

    def correction(self, fneq, xi, w, Phi, P):
        """delta f [Q, N] from the streamed non-equilibrium populations [Q, N]."""
        z = (Phi @ fneq).T
        o, _ = self.forward(z * self.s_in)
        return (w[:, None] * self.sigma) * (P @ o.T)


def bf16_round(a):
    """Round float64 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
