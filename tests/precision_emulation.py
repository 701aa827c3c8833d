"""Error models of the split chain's product arithmetic, for tests only: numbers are split into
pieces with a short mantissa (TF32: 10 explicit bits, BF16: 7), the pieces' cross products are
accumulated in FP32, and the chain's intermediates are FP32.  Used to bound the split path's error
on rough data and to decide between split precisions; never a reference result.

Accumulation: "rn" rounds the FP32 accumulator to nearest after each product; "rz8" models the
tensor cores' truncating accumulation: every 8-wide K step of every piece product (one tcgen05 MMA
of kind tf32) adds its exact partial sum to the accumulator, which is then rounded toward zero to
FP32."""
import numpy as np

from oracle.phi import phi1
from oracle.stepper import rhs


def round_mantissa(x, bits):
    """Round FP32 values to `bits` explicit mantissa bits (to nearest, ties away from zero)."""
    a = np.asarray(x, dtype=np.float32).view(np.uint32)
    drop = 23 - bits
    mask = np.uint32((0xFFFFFFFF << drop) & 0xFFFFFFFF)
    return ((a + np.uint32(1 << (drop - 1))) & mask).astype(np.uint32).view(np.float32)


def pieces(x, bits, count):
    out, r = [], np.asarray(x, dtype=np.float32)
    for _ in range(count):
        p = round_mantissa(r, bits)
        out.append(p)
        r = (r - p).astype(np.float32)
    return out


SCHEMES = {
    # name: (mantissa bits, pieces, cross products (i, j) kept, smallest first)
    "tf32x3": (10, 2, [(0, 1), (1, 0), (0, 0)]),
    "bf16x3": (7, 2, [(0, 1), (1, 0), (0, 0)]),
    "bf16x6": (7, 3, [(0, 2), (2, 0), (1, 1), (0, 1), (1, 0), (0, 0)]),
}


def _rz32(x):
    """FP64 values rounded toward zero to FP32 (returned as FP64)."""
    r = np.asarray(x, dtype=np.float64).astype(np.float32)
    bad = np.abs(r.astype(np.float64)) > np.abs(x)
    if np.any(bad):
        r[bad] = np.nextafter(r[bad], np.float32(0))
    return r.astype(np.float64)


def matmul(A, B, scheme="tf32x3", accumulate="rn"):
    """A @ B with the scheme's split products accumulated in FP32 (see the module docstring)."""
    bits, count, terms = SCHEMES[scheme]
    a, b = pieces(A, bits, count), pieces(B, bits, count)
    if accumulate == "rn":
        acc = np.zeros(np.shape(A)[:-1] + (np.shape(B)[-1],), np.float32)
        for i, j in terms:
            acc = (acc + (a[i] @ b[j])).astype(np.float32)
        return acc.astype(np.float64)
    a = [x.astype(np.float64) for x in a]
    b = [x.astype(np.float64) for x in b]
    K = np.shape(A)[-1]
    acc = np.zeros(np.shape(A)[:-1] + (np.shape(B)[-1],))
    for k0 in range(0, K, 8):
        ks = slice(k0, min(K, k0 + 8))
        for i, j in terms:
            acc = _rz32(acc + a[i][..., ks] @ b[j][ks, :])
    return acc


def f32(x):
    return np.asarray(x).astype(np.float32).astype(np.float64)


def advance(problem, W, F, scheme="tf32x3", accumulate="rn", plain=()):
    """w + tau phi_1 ... phi_1 F with F and every intermediate in FP32 and every product in the scheme.
    Modes in `plain` are applied as one product with the matrix phi_1(tau d A_mu) (formed in FP64), the
    others through their eigenbasis (two products and the FP32 Hadamard factor)."""
    g = problem.grid
    out = np.array(W, copy=True)
    for s in range(problem.S):
        X = f32(F[s])
        for mu in range(g.ndim, 0, -1):
            lam, V, Vinv = problem._eig[mu]
            axis = X.ndim - mu
            t = problem.tau * problem.d[s]
            if mu in plain:
                P = (V * phi1(t * lam)[None, :]) @ Vinv
                X = np.moveaxis(matmul(np.moveaxis(X, axis, -1), P.T, scheme, accumulate), -1, axis)
                continue
            sc = np.moveaxis(np.broadcast_to(g.scale[mu], X.shape), axis, -1)[..., :1]
            Z = matmul(np.moveaxis(X, axis, -1), Vinv.T, scheme, accumulate)
            Z = f32(f32(Z) * f32(phi1(t * sc * lam)))
            X = np.moveaxis(matmul(Z, V.T, scheme, accumulate), -1, axis)
        out[s] = W[s] + f32(problem.tau * X)
    return out


def run(problem, W0, steps, scheme="tf32x3", accumulate="rn", plain=()):
    W = np.array(W0, copy=True)
    for _ in range(steps):
        W = advance(problem, W, rhs(problem, W), scheme, accumulate, plain)
    return W
