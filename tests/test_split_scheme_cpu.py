"""The split-precision scheme's accuracy from its arithmetic alone (CPU, no GPU): an emulation in
numpy of the Ozaki splitting (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012) as the
split path applies it to the Hamiltonian contraction h = E^T D E of each batch (Eq.
batch_matrix_mult): every row of F = E sqrt|D| is scaled by a power of two 2^-e with
max |x 2^-e| in [1/4, 1/2), cut into S balanced base-64 digits (|d| <= 32, exact in bf16), and the
slice products D_s D_t^T are summed exactly for s + t < S (the pairs with s + t >= S carry a
weight below 64^-S and are dropped); negative weights flip the sign of the B operand's columns.

The density's T = Phi P is split the same way with one exponent per point (row of Phi) and
one per batch (its block of P); the local Pulay matrix elements, for which no kernel exists yet,
as a non-symmetric product with one exponent per row of each operand.

The emulation takes the oracle's basis functions, so it checks the scheme and the tolerance the
split path is held to, not the kernels (the GPU tests do that): the error against the FP64
results falls about 64^2 per two slices, and 10 slices meet the 1e-10 bar for H and n on the
water molecule (with the metric of tests/_metrics.py)."""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_1912_06636_gb300 import synth
from tests._metrics import rel_err


def _split_product(F, sign, S):
    """Emulated sum over s + t < S of (digits_s of F)(sign * digits_t of F)^T, scaled back."""
    mx = np.abs(F).max(axis=1)
    e = np.array([math.frexp(m)[1] + 1 if m > 0 else 0 for m in mx], dtype=np.int64)  # m 2^-e in [1/4, 1/2)
    r = F * np.exp2(-e.astype(np.float64))[:, None]
    digits = []
    for _ in range(S):
        t = r * 64.0
        d = np.rint(t)  # balanced digit, |d| <= 32
        digits.append(d)
        r = t - d
    acc = np.zeros((F.shape[0], F.shape[0]))
    for s in range(S):
        for t in range(S - s):
            # exact: |d| <= 32 and K < 2^33, so every integer sum is below 2^53
            acc += (digits[s] @ (digits[t] * sign[None, :]).T) * 2.0 ** (-6 * (s + t + 2))
    return acc * np.exp2((e[:, None] + e[None, :]).astype(np.float64))


@pytest.fixture(scope="module")
def water_batches():
    s = synth.config_water()
    o = Oracle(s)
    v = s.potential()
    off, perm = Oracle.partition(s.pt_xyz, 200)
    ro, ri = o.relevance(s.pt_xyz, off, perm)
    out = []
    for b in range(len(off) - 1):
        rel = ri[ro[b]:ro[b + 1]]
        if len(rel) == 0:
            continue
        idx = perm[off[b]:off[b + 1]]
        phi, grad = o.eval_dense(s.pt_xyz[idx])
        E = np.concatenate([phi[:, rel].T] + [grad[:, rel, c].T for c in range(3)], axis=1)
        w = s.pt_w[idx]
        d = np.concatenate([w * v[idx], 0.5 * w, 0.5 * w, 0.5 * w])
        out.append((rel, E, d))
    return s.n_basis, out


def test_split_error_per_slice_count(water_batches):
    nb, batches = water_batches
    ref, A = np.zeros((nb, nb)), np.zeros((nb, nb))
    emu = {S: np.zeros((nb, nb)) for S in (4, 6, 8, 10)}
    for rel, E, d in batches:
        ix = np.ix_(rel, rel)
        ref[ix] += (E * d[None, :]) @ E.T
        A[ix] += np.abs(E * d[None, :]) @ np.abs(E).T
        F = E * np.sqrt(np.abs(d))[None, :]
        sign = np.where(d < 0, -1.0, 1.0)
        for S in emu:
            emu[S][ix] += _split_product(F, sign, S)
    err = {S: rel_err(emu[S], ref, A) for S in emu}
    print({S: f"{e:.2e}" for S, e in err.items()})
    assert err[4] > 1e-8  # the test is not vacuous
    for S in (4, 6):
        assert err[S] / max(err[S + 2], 1e-300) > 500.0  # about 64^2 per two slices
    assert err[10] <= 1e-10


def _split_matmul(X, ex, Y, ey, S):
    """Emulated split product X Y with per-row exponents ex of X and one exponent ey for all of Y
    (the density's T = Phi P: exponents per point and per batch)."""
    def digits(M, scale):
        r = M * scale
        out = []
        for _ in range(S):
            t = r * 64.0
            d = np.rint(t)
            out.append(d)
            r = t - d
        return out

    dx = digits(X, np.exp2(-ex.astype(np.float64))[:, None])
    dy = digits(Y, 2.0 ** -ey)
    acc = np.zeros((X.shape[0], Y.shape[1]))
    for s in range(S):
        for t in range(S - s):
            acc += (dx[s] @ dy[t]) * 2.0 ** (-6 * (s + t + 2))
    return acc * np.exp2(ex.astype(np.float64))[:, None] * 2.0 ** ey


def _exponent(m):
    return math.frexp(m)[1] + 1 if m > 0 else 0


def test_split_density_error_per_slice_count():
    """The density n_q = sum_j T_qj phi_qj with T = Phi P split (Eq. Density), P of the water
    molecule (seed 0): the error against the oracle falls about 64^2 per two slices and 10
    slices meet 1e-10 with the metric of tests/_metrics.py."""
    s = synth.config_water()
    o = Oracle(s)
    P = synth.density_matrix(s, 0)
    nref, D, _ = o.density(s.pt_xyz, P, s.pt_w)
    off, perm = Oracle.partition(s.pt_xyz, 200)
    ro, ri = o.relevance(s.pt_xyz, off, perm)
    emu = {S: np.zeros(s.n_points) for S in (4, 6, 8, 10)}
    for b in range(len(off) - 1):
        rel = ri[ro[b]:ro[b + 1]]
        if len(rel) == 0:
            continue
        idx = perm[off[b]:off[b + 1]]
        phi, _ = o.eval_dense(s.pt_xyz[idx])
        Phi = phi[:, rel]
        Pb = P[np.ix_(rel, rel)]
        ex = np.array([_exponent(m) for m in np.abs(Phi).max(axis=1)], dtype=np.int64)
        ey = _exponent(np.abs(Pb).max())
        for S in emu:
            T = _split_matmul(Phi, ex, Pb, ey, S)
            emu[S][idx] = np.sum(T * Phi, axis=1)
    err = {S: rel_err(emu[S], nref, D) for S in emu}
    print({S: f"{e:.2e}" for S, e in err.items()})
    assert err[4] > 1e-8
    for S in (4, 6):
        assert err[S] / max(err[S + 2], 1e-300) > 500.0
    assert err[10] <= 1e-10


def _rint_small(y):
    # rint of |y| < 2^22 by adding and subtracting 1.5 2^23 in FP32 (the kernels' rounding)
    c = np.float32(12582912.0)
    return np.float32(np.float32(y + c) - c)


def _part_chunks(P, CB):
    """The slicers' top-down FP32 chunking of one scaled part P (an FP32 value): q_c =
    rint(R 2^-(c CB)), R <- R - q_c 2^(c CB) for c = 3, 2, 1, then u_0 = rint(R). The FMA
    R - q 2^(c CB) is emulated in FP64, where it is exact, then rounded to FP32."""
    R = np.float32(P)
    out = [0.0] * 4
    for c in (3, 2, 1):
        q = _rint_small(np.float32(R * np.float32(2.0 ** (-c * CB))))
        R = np.float32(np.float64(R) - np.float64(q) * 2.0 ** (c * CB))
        out[c] = q
    out[0] = _rint_small(R)
    return out


@pytest.mark.parametrize("B,S", [(5, 8), (5, 14), (5, 16), (6, 4), (6, 10), (6, 12)])
def test_float_float_chunks_are_exact(B, S):
    """Digits of a float-float value x = h + l (the split path's evaluation) come from balanced
    CB-bit chunks of round(h 2^(BS-e)) + round(l 2^(BS-e)), formed in FP32 without integer
    arithmetic: every chunk is an exact integer of at most 2^CB in magnitude and the chunks sum
    exactly to that integer (checked against Python's exact integers, ties aside), for values
    spread over 60 binades below the row's bound |x 2^-e| < 1/2."""
    from fractions import Fraction

    rng = np.random.default_rng(B * 100 + S)
    D = 3 if B == 6 else 4
    CB, BS = D * B, B * S
    for _ in range(3000):
        e = int(rng.integers(-60, 60))
        x = rng.uniform(-0.5, 0.5) * 2.0 ** (-int(rng.integers(0, 60))) * 2.0 ** e
        h = np.float32(x)
        lo = np.float32(x - np.float64(h))
        H = np.float32(np.float64(h) * 2.0 ** (BS - e))
        L = np.float32(np.float64(lo) * 2.0 ** (BS - e))
        u = [a + b for a, b in zip(_part_chunks(H, CB), _part_chunks(L, CB))]
        assert all(float(c) == int(c) and abs(c) <= 2 ** CB for c in u)
        X = sum(int(u[c]) << (c * CB) if u[c] >= 0 else -((-int(u[c])) << (c * CB)) for c in range(4))
        ref = round(Fraction(float(H))) + round(Fraction(float(L)))
        assert abs(X - ref) <= 1
        assert abs(X) < 2 ** (BS - 1) + 2


def _split_general(X, Y, S):
    """Emulated split product X Y^T with one exponent per row of X and per row of Y (no sign
    flips: the weights sit in Y), base-64 digits, the pairs s + t < S."""
    def digits(M):
        mx = np.abs(M).max(axis=1)
        e = np.array([_exponent(m) for m in mx], dtype=np.int64)
        r = M * np.exp2(-e.astype(np.float64))[:, None]
        out = []
        for _ in range(S):
            t = r * 64.0
            d = np.rint(t)
            out.append(d)
            r = t - d
        return out, e

    dx, ex = digits(X)
    dy, ey = digits(Y)
    acc = np.zeros((X.shape[0], Y.shape[0]))
    for s in range(S):
        for t in range(S - s):
            acc += (dx[s] @ dy[t].T) * 2.0 ** (-6 * (s + t + 2))
    return acc * np.exp2((ex[:, None] + ey[None, :]).astype(np.float64))


def test_split_pulay_products_per_slice_count():
    """The local Pulay matrix elements as split products (the split path's next step, no kernel
    yet): M^c = (d_c Phi)^T W (-1/2 lap + v) Phi and S^c = (d_c Phi)^T W Phi per batch, with
    separate digit sets for the two operands (the products are not symmetric) and one exponent
    per operand row. On water the error against the oracle's matrices, measured against their
    magnitude sums, falls about 64^2 per two slices, as for H, and 10 slices meet 1e-10."""
    s = synth.config_water()
    o = Oracle(s)
    v = s.potential()
    Mref, Sref, AM, AS = o.pulay_matrices(s.pt_xyz, s.pt_w, v)
    off, perm = Oracle.partition(s.pt_xyz, 200)
    ro, ri = o.relevance(s.pt_xyz, off, perm)
    nb = s.n_basis
    emuM = {S: np.zeros((3, nb, nb)) for S in (6, 8, 10)}
    emuS = {S: np.zeros((3, nb, nb)) for S in (6, 8, 10)}
    for b in range(len(off) - 1):
        rel = ri[ro[b]:ro[b + 1]]
        if len(rel) == 0:
            continue
        idx = perm[off[b]:off[b + 1]]
        phi, grad, hess = o.eval_dense2(s.pt_xyz[idx])
        lap = hess[:, :, 0] + hess[:, :, 3] + hess[:, :, 5]
        w = s.pt_w[idx][:, None]
        hphi = (w * (-0.5 * lap[:, rel] + v[idx][:, None] * phi[:, rel])).T   # [N, P]
        wphi = (w * phi[:, rel]).T
        ix = np.ix_(rel, rel)
        for c in range(3):
            A = grad[:, rel, c].T
            for S in emuM:
                emuM[S][c][ix] += _split_general(A, hphi, S)
                emuS[S][c][ix] += _split_general(A, wphi, S)
    err = {S: max(rel_err(emuM[S], Mref, AM), rel_err(emuS[S], Sref, AS)) for S in emuM}
    print({S: f"{e:.2e}" for S, e in err.items()})
    assert err[6] > 1e-12
    assert err[6] / max(err[8], 1e-300) > 500.0
    assert err[10] <= 1e-10
