"""Counter-based Gaussian stream of the oracle (plain NumPy, FP64).

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

The paper draws its test matrices Phi_j / Psi_j "with i.i.d. standard Gaussian
entries" (Sec. 3.2, Algorithm 2 and the one-pass variant after Theorem 3.3)
but does not say how; this library fixes a counter-based stream so that the
test matrices can be regenerated on demand instead of stored.

Definition (written here from the published algorithm, independently of the
CUDA side, which implements the same definition in its own code):

* Philox4x32-10 of Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
  easy as 1, 2, 3" (SC'11): 10 rounds; each round multiplies counter words 0 and
  2 by 0xD2511F53 and 0xCD9E8D57 (32x32 -> 64-bit), and the new counter is
  (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); after each round the key is bumped
  by (0x9E3779B9, 0xBB67AE85) modulo 2^32.
* key = (seed mod 2^32, seed div 2^32).
* Entry (row, j) of the test matrix with stream id s uses the counter
  (row mod 2^32, row div 2^32, j div 4, s); the four output words (x0..x3)
  give four normals by Box-Muller:
      u(x) = (x + 1/2) 2^-32,
      rho_a = sqrt(-2 ln u(x0)),  theta_a = 2 pi u(x1)
      rho_b = sqrt(-2 ln u(x2)),  theta_b = 2 pi u(x3)
      z_{4q+0} = rho_a cos theta_a,  z_{4q+1} = rho_a sin theta_a,
      z_{4q+2} = rho_b cos theta_b,  z_{4q+3} = rho_b sin theta_b.
* Stream ids: the right test matrix Omega_k of unfolding k (column sketch) is
  s = k; the left test matrix Psi_k (row sketch) is s = 64 + k.

Khatri-Rao test matrices (Sec. 3.2, the substitute for dense Phi_j that the
paragraph after Theorem 3.3 describes, eq. (sketch_orig)): the test matrix of
one sketch is a row-wise Khatri-Rao product of small i.i.d. Gaussian factors,
one per mode its rows run over.  Here the factor of mode m (1-based) of the
sketch with stream s is the n_m x l matrix whose row i is row
i + (2^31 + m) 2^32 of stream s (the row-high word has its top bit set, so no
factor row coincides with a row of a dense test matrix), and the entry of the
product at the column-major multi-index (i_{m_1}, i_{m_2}, ...) (first listed
mode fastest, modes in increasing order) is
    F_{m_1}(i_{m_1}, j) * F_{m_2}(i_{m_2}, j) * ...
(rounding order: increasing modes for a column sketch's Omega_k, decreasing
for a row sketch's Psi_k; in FP64 the order changes the last bit only).  The paper writes the product Psi_d (.) ... (.)
Psi_{j+1} for the column space of X_j; with the Kronecker convention of the
Khatri-Rao product (the last factor's index fastest) its rows run over
(i_{j+1}, ..., i_d) column-major, the column index of X_j.
"""
import numpy as np

PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)
_SH32 = np.uint64(32)

STREAM_OMEGA = 0    # + k
STREAM_PSI = 64     # + k


def philox4x32_10(c0, c1, c2, c3, key0, key1):
    """Philox4x32-10 on arrays of 32-bit counter words (held in uint64).

    Returns the four output words as uint64 arrays holding 32-bit values.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = int(key0) & 0xFFFFFFFF
    k1 = int(key1) & 0xFFFFFFFF
    for _ in range(10):
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> _SH32, p0 & _MASK32
        hi1, lo1 = p1 >> _SH32, p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                          hi0 ^ c3 ^ np.uint64(k1), lo0)
        k0 = (k0 + PHILOX_W0) & 0xFFFFFFFF
        k1 = (k1 + PHILOX_W1) & 0xFFFFFFFF
    return c0, c1, c2, c3


def _uniform(x):
    return (x.astype(np.float64) + 0.5) * 2.0 ** -32


def gaussian(seed, stream, rows, ncols):
    """Rows `rows` (array of indices) and columns 0..ncols-1 of a test matrix.

    Returns an array of shape (len(rows), ncols) in FP64.
    """
    rows = np.asarray(rows, dtype=np.uint64).ravel()
    seed = int(seed)
    k0, k1 = seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF
    out = np.empty((rows.size, ncols), dtype=np.float64)
    lo, hi = rows & _MASK32, rows >> _SH32
    for q in range((ncols + 3) // 4):
        x0, x1, x2, x3 = philox4x32_10(lo, hi, np.uint64(q), np.uint64(stream), k0, k1)
        rho_a = np.sqrt(-2.0 * np.log(_uniform(x0)))
        th_a = 2.0 * np.pi * _uniform(x1)
        rho_b = np.sqrt(-2.0 * np.log(_uniform(x2)))
        th_b = 2.0 * np.pi * _uniform(x3)
        zs = (rho_a * np.cos(th_a), rho_a * np.sin(th_a),
              rho_b * np.cos(th_b), rho_b * np.sin(th_b))
        for t in range(4):
            j = 4 * q + t
            if j < ncols:
                out[:, j] = zs[t]
    return out


def test_matrix(seed, stream, nrows, ncols):
    """The full nrows x ncols test matrix of one stream (dense, FP64)."""
    return gaussian(seed, stream, np.arange(nrows, dtype=np.uint64), ncols)


KR_ROW_HI = 0x80000000


def kr_factor(seed, stream, mode, n, ncols):
    """Gaussian factor of mode `mode` (1-based) of a Khatri-Rao test matrix:
    n x ncols, row i = row i + (2^31 + mode) 2^32 of the stream."""
    base = np.uint64((KR_ROW_HI + int(mode)) << 32)
    return gaussian(seed, stream, np.arange(n, dtype=np.uint64) + base, ncols)


def kr_test_matrix(seed, stream, modes, sizes, ncols, decreasing=False):
    """The Khatri-Rao test matrix over `modes` (increasing, 1-based) of sizes
    `sizes`: prod(sizes) x ncols, row = column-major multi-index with the first
    mode fastest, entry = product of the factor entries (FP64), multiplied in
    increasing mode order (decreasing=True: decreasing order).  This is the
    dense form of F_{m_last} (.) ... (.) F_{m_1}."""
    Fs = [kr_factor(seed, stream, m, n, ncols) for m, n in zip(modes, sizes)]
    if not decreasing:
        out = np.ones((1, ncols))
        for F in Fs:
            # rows of the product so far are the faster index: new row = r + R i
            out = (out[None, :, :] * F[:, None, :]).reshape(-1, ncols)
        return out
    out = np.ones((1, ncols))
    for F in reversed(Fs):
        # the product so far runs over the slower modes: new row = i + n r
        out = (F[None, :, :] * out[:, None, :]).reshape(-1, ncols)
    return out


def round_to(a, fmt):
    """Round FP64 values to a narrower floating format, nearest-even.

    fmt: 'f64' (identity), 'f32', 'tf32' (8-bit exponent, 10-bit mantissa),
    'bf16' (8-bit exponent, 7-bit mantissa) or 'fp16' (IEEE binary16: 5-bit
    exponent, 10-bit mantissa, subnormals below 2^-14, magnitudes that round
    above 65504 become infinite).  The value is first held in FP32 (as the
    product path holds it), then rounded once.  Used by tests that mirror the
    precision of a mixed-precision product path on the oracle side.
    """
    a = np.asarray(a, dtype=np.float64)
    if fmt == 'f64':
        return a.copy()
    f = a.astype(np.float32)
    if fmt == 'f32':
        return f.astype(np.float64)
    if fmt == 'fp16':
        return _round_binary16(f.astype(np.float64))
    drop = {'tf32': 13, 'bf16': 16}[fmt]
    u = f.view(np.uint32).astype(np.uint64)
    half = np.uint64(1 << (drop - 1))
    lsb = (u >> np.uint64(drop)) & np.uint64(1)
    u = (u + half - np.uint64(1) + lsb) & ~np.uint64((1 << drop) - 1)
    return (u & _MASK32).astype(np.uint32).view(np.float32).astype(np.float64)


def _round_binary16(v):
    """Nearest-even rounding of FP64 values to IEEE binary16, from the format:
    the quantum of a value is 2^(e - 10) with e its binary exponent, clamped
    below at -14 (the subnormal range has the fixed quantum 2^-24); the largest
    finite value is 65504 = (2 - 2^-10) 2^15, and a result above it is an
    overflow (infinite).  Infinities and NaNs pass through."""
    v = np.asarray(v, dtype=np.float64)
    out = v.copy()
    fin = np.isfinite(v) & (v != 0.0)
    m, e = np.frexp(np.abs(v[fin]))           # |v| = m 2^e, m in [0.5, 1)
    q = np.ldexp(1.0, np.maximum(e - 1, -14) - 10)
    r = np.round(v[fin] / q) * q               # exact scaling; np.round is half-to-even
    r[np.abs(r) > 65504.0] = np.inf * np.sign(r[np.abs(r) > 65504.0])
    out[fin] = r
    return out
