"""Gauge-covariant convolutional preconditioner, oracle form (numpy FP64).

Not from the paper (which has no learned component); it is the learned
smoother of this library, defined here so that the CUDA kernels can be checked
against a plain implementation.  Test infrastructure only.

Definition
  transporters  T_d(x) for the 9 offsets d = (dx, dt) in {-1,0,1}^2, carrying a
                field from x + d to x:  T_(0,0) = 1, T_(+1,0) = U_0(x),
                T_(-1,0) = conj(U_0(x - e0)), T_(0,+1) = U_1(x), T_(0,-1) =
                conj(U_1(x - e1)), each t-link that crosses the time boundary
                with a factor -1 (antiperiodic fermions); the diagonals average
                the two L-shaped paths:
                  T_(a,b)(x) = 1/2 [T_(a,0)(x) T_(0,b)(x + a e0) + T_(0,b)(x) T_(a,0)(x + b e1)].
                Under a gauge transformation psi -> Omega psi, U_mu(x) ->
                Omega(x) U_mu(x) conj(Omega(x + mu)) every T_d(x) picks up
                Omega(x) conj(Omega(x + d)), so the layers below are covariant.
  layer l       z(x)_c' = sum_d sum_c W_l[d][c'][c] T_d(x) a(x + d)_c
                a'(x)_c' = z * max(0, |z| + b_c') / |z|  (hidden layers; |z| = 0 -> 0)
                the last layer is linear.  Channels: 2 (spin) -> C -> ... -> C -> 2.
  weights       complex W_l[9][c_out][c_in] used rounded to bfloat16 (each real and
                imaginary part, round to nearest even), real biases b_l[c_out] (FP32).
  loss          (1/nrhs) sum_r ||M(r_r) - e_r||^2 / ||e_r||^2.
  gradients     for a real loss and complex z, g = dL/dRe z + i dL/dIm z:
                y = W u  ->  g_W += g_y conj(u),  g_u += conj(W) g_y.
Offsets are enumerated d = 3 * (dt + 1) + (dx + 1).
Arrays: fields a[nrhs, L*L, C] (site = t * L + x), links U[t, x, mu].

Tensor-core number format (tc=True), the arithmetic of the library's tcgen05 layers with BF16 operands:
  forward       every layer input a (the residual r included) is rounded to bfloat16 (real and imaginary
                parts) before the channel mixing; the mixing sums, transports, activation and the output
                stay exact here (FP32 in the library).
  backward      the gradient w.r.t. each layer's pre-activation, gz, is rounded to bfloat16 before it enters
                the weight gradient and the input gradient; the transported inputs u = T_d a are rounded to
                bfloat16 for the weight gradient.  The rounding steps are passed through unchanged in the
                derivative (the gradient is that of the same formulas without them).
  The library's input gradient uses the identity conj(T_d(y - d)) = T_(-d)(y) (the reversed path), so it
  is the same gathered mixing as the forward with the weights conj(W[-d])^T; that identity is pinned by the
  tests of this module.
"""
from __future__ import annotations

import numpy as np

OFFSETS = [(dx, dt) for dt in (-1, 0, 1) for dx in (-1, 0, 1)]


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 (ties to even), via float32 bits."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def round_weights(W: np.ndarray) -> np.ndarray:
    return bf16_round(W.real) + 1j * bf16_round(W.imag)


def bf16_complex(a: np.ndarray) -> np.ndarray:
    """Real and imaginary parts rounded to the nearest bfloat16."""
    return bf16_round(np.real(a)) + 1j * bf16_round(np.imag(a))


def transporters(U: np.ndarray) -> np.ndarray:
    """T[site, d] complex128 for the 9 offsets."""
    L = U.shape[0]
    t = np.arange(L)[:, None] * np.ones((1, L), int)
    sgn_f = np.where(t == L - 1, -1.0, 1.0)   # t-link from t to t+1 crossing the boundary
    U0 = U[..., 0]
    U1 = U[..., 1] * sgn_f

    def sh(a, dx, dt):   # a(x + d) as an array over x
        return np.roll(np.roll(a, -dt, axis=0), -dx, axis=1)

    Tx = {0: np.ones((L, L), complex), 1: U0, -1: np.conj(sh(U0, -1, 0))}
    Tt = {0: np.ones((L, L), complex), 1: U1, -1: np.conj(sh(U1, 0, -1))}
    out = np.empty((L * L, 9), complex)
    for d, (dx, dt) in enumerate(OFFSETS):
        if dx == 0 or dt == 0:
            T = Tx[dx] * Tt[dt]
        else:
            T = 0.5 * (Tx[dx] * sh(Tt[dt], dx, 0) + Tt[dt] * sh(Tx[dx], 0, dt))
        out[:, d] = T.ravel()
    return out


def neighbour_index(L: int) -> np.ndarray:
    """nb[site, d] = index of site + d (periodic)."""
    t, x = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    nb = np.empty((L * L, 9), int)
    for d, (dx, dt) in enumerate(OFFSETS):
        nb[:, d] = (((t + dt) % L) * L + (x + dx) % L).ravel()
    return nb


class Net:
    def __init__(self, U, weights, biases, round_bf16=True, tc=False):
        """weights: list of complex arrays [9, c_out, c_in]; biases: list (len = layers - 1) of real [c_out];
        tc: the tensor-core number format (module docstring)."""
        self.L = U.shape[0]
        self.tc = tc
        self.T = transporters(U)
        self.nb = neighbour_index(self.L)
        self.W = [round_weights(w) if round_bf16 else np.asarray(w, complex) for w in weights]
        self.b = [np.asarray(b, float) for b in biases]

    def _gather(self, a):
        # u[r, x, d, c] = T_d(x) a[r, x + d, c]
        return self.T[None, :, :, None] * a[:, self.nb, :]

    def forward(self, r):
        """r[nrhs, V, 2] -> output [nrhs, V, 2]; keeps the tape for backward."""
        self.tape = []
        a = r
        for l, W in enumerate(self.W):
            if self.tc:
                a = bf16_complex(a)
            u = self._gather(a)
            z = np.einsum("dkc,rxdc->rxk", W, u)
            if l < len(self.W) - 1:
                mag = np.abs(z)
                s = np.where(mag > 0, np.maximum(0.0, mag + self.b[l][None, None, :]) / np.where(mag > 0, mag, 1), 0)
                a_next = z * s
            else:
                a_next = z
            self.tape.append((a, u, z))
            a = a_next
        return a

    def loss(self, r, e):
        y = self.forward(r)
        en = np.sum(np.abs(e) ** 2, axis=(1, 2))
        return float(np.mean(np.sum(np.abs(y - e) ** 2, axis=(1, 2)) / en)), y

    def backward(self, r, e):
        """Loss and gradients (dL/dRe + i dL/dIm for W, dL/db for b)."""
        L_, y = self.loss(r, e)
        nr = r.shape[0]
        en = np.sum(np.abs(e) ** 2, axis=(1, 2))
        g = 2.0 * (y - e) / (nr * en[:, None, None])
        gW = [None] * len(self.W)
        gb = [None] * len(self.b)
        for l in range(len(self.W) - 1, -1, -1):
            a, u, z = self.tape[l]
            if l < len(self.W) - 1:   # activation backward
                mag = np.abs(z)
                on = (mag + self.b[l][None, None, :]) > 0
                ph = np.where(mag > 0, z / np.where(mag > 0, mag, 1), 0)
                rad = np.real(np.conj(ph) * g)
                scale = np.where(mag > 0, (mag + self.b[l][None, None, :]) / np.where(mag > 0, mag, 1), 0)
                gz = np.where(on, rad * ph + scale * (g - rad * ph), 0)
                gb[l] = np.sum(np.where(on, rad, 0), axis=(0, 1))
            else:
                gz = g
            if self.tc:
                gz = bf16_complex(gz)
                u = bf16_complex(u)
            gW[l] = np.einsum("rxk,rxdc->dkc", gz, np.conj(u))
            gu = np.einsum("dkc,rxk->rxdc", np.conj(self.W[l]), gz)
            # u = T_d(x) a(x + d): g_a(y) += conj(T_d(x)) g_u(x, d) for y = x + d
            ga = np.zeros_like(a)
            contrib = np.conj(self.T)[None, :, :, None] * gu
            for d in range(9):
                np.add.at(ga, (slice(None), self.nb[:, d], slice(None)), contrib[:, :, d, :])
            g = ga
        return L_, gW, gb


def init_params(channels: int, layers: int, seed: int):
    """Deterministic initial weights (scaled complex Gaussian) and zero biases (numpy PCG64)."""
    rs = np.random.default_rng(seed)
    dims = [2] + [channels] * (layers - 1) + [2]
    W, b = [], []
    for l in range(layers):
        ci, co = dims[l], dims[l + 1]
        s = 1.0 / np.sqrt(9 * ci)
        W.append(s * (rs.standard_normal((9, co, ci)) + 1j * rs.standard_normal((9, co, ci))) / np.sqrt(2))
        if l < layers - 1:
            b.append(np.zeros(co))
    return W, b
