"""The FMM operators in the scaled form the CUDA kernels use (Section 3.2.1;
Greengard-Rokhlin expansions of the field E(z) = sum_j q_j / (z - z_j),
F_rep(i) = kr m_i conj(E(z_i))), each checked against the direct sum on
random clusters, in FP64 on the CPU.

Coefficients are scaled by the box half-width r: outgoing a~_k = a_k / r^k,
incoming b~_l = b_l r^l.  Boxes of one level are 2r wide, so the centre
offset of a V-list pair is r w with w = 2 (dx + i dy) for integer cell
offsets (dx, dy) in [-3, 3]^2, max(|dx|, |dy|) >= 2: the M2L matrix of a
class depends on w only.  Every truncation error below is bounded by a
geometric series in the ratio of the cluster radius to the distance, so
each test asks for that bound and checks that the error falls with p.
These pins hold the formulas; the GPU kernels that apply them are checked
end to end against the exact sum in tests/test_gpu_fmm.py."""
import math

import numpy as np
import pytest

C = math.comb


def cluster(rng, c, r, n):
    """n charges uniform in the square of half-width r around c."""
    z = c + r * (rng.uniform(-1, 1, n) + 1j * rng.uniform(-1, 1, n))
    q = rng.uniform(0.5, 2.0, n)
    return z, q


def direct(zt, zs, q):
    return np.array([np.sum(q / (z - zs)) for z in zt])


def p2m(zs, q, c, r, p):
    """a~_0 = sum q, a~_k = -sum q ((z_j - c) / r)^k / k."""
    w = (zs - c) / r
    a = np.zeros(p + 1, complex)
    a[0] = q.sum()
    for k in range(1, p + 1):
        a[k] = -np.sum(q * w ** k) / k
    return a


def m2p(a, c, r, z):
    """E(z) = (a~_0 - sum_k k a~_k t^k) / (z - c), t = r / (z - c)."""
    t = r / (z - c)
    s = sum(k * a[k] * t ** k for k in range(1, len(a)))
    return (a[0] - s) / (z - c)


def m2m(a, c_old, r_old, c_new, r_new):
    """Unscaled b_l = -a_0 z0^l / l + sum_{k=1..l} a_k z0^(l-k) C(l-1, k-1), z0 = c_old - c_new."""
    p = len(a) - 1
    au = np.array([a[k] * r_old ** k for k in range(p + 1)])
    z0 = c_old - c_new
    b = np.zeros(p + 1, complex)
    b[0] = au[0]
    for l in range(1, p + 1):
        b[l] = -au[0] * z0 ** l / l + sum(au[k] * z0 ** (l - k) * C(l - 1, k - 1) for k in range(1, l + 1))
    return np.array([b[l] / r_new ** l for l in range(p + 1)])


def m2l_class(a, w):
    """b~_l = w^-l (-a~_0 / l + sum_k (-1)^k a~_k w^-k C(l+k-1, k-1)), l >= 1 (b~_0 unused)."""
    p = len(a) - 1
    b = np.zeros(p + 1, complex)
    for l in range(1, p + 1):
        s = -a[0] / l + sum((-1) ** k * a[k] * w ** (-k) * C(l + k - 1, k - 1) for k in range(1, p + 1))
        b[l] = s * w ** (-l)
    return b


def p2l(zs, q, c, r, p):
    """b~_l = -sum q t^l / l, t = r / (z_j - c), l >= 1."""
    t = r / (zs - c)
    b = np.zeros(p + 1, complex)
    for l in range(1, p + 1):
        b[l] = -np.sum(q * t ** l) / l
    return b


def l2p(b, c, r, z):
    """E(z) = (1/r) sum_l l b~_l v^(l-1), v = (z - c) / r."""
    v = (z - c) / r
    return sum(l * b[l] * v ** (l - 1) for l in range(1, len(b))) / r


def l2l_fold(b, t, D):
    """Shift of an ancestor's expansion (half-width r_A) to a descendant D
    levels finer: b~_m += 2^(-D m) sum_{l >= m} b~_l C(l, m) t^(l - m),
    t = (c_leaf - c_A) / r_A."""
    p = len(b) - 1
    out = np.zeros(p + 1, complex)
    for m in range(1, p + 1):
        out[m] = 2.0 ** (-D * m) * sum(b[l] * C(l, m) * t ** (l - m) for l in range(m, p + 1))
    return out


def rel(x, y):
    return np.max(np.abs(x - y)) / np.max(np.abs(y))


RHO_V = math.sqrt(2) / (4 - math.sqrt(2))     # V-list geometry


def test_p2m_m2p_against_direct():
    rng = np.random.default_rng(1)
    c, r = 0.3 - 0.2j, 0.5
    zs, q = cluster(rng, c, r, 200)
    zt = c + 3.0 * np.exp(2j * np.pi * rng.uniform(0, 1, 50))     # |z - c| = 3: ratio sqrt(2) r / 3
    ex = direct(zt, zs, q)
    rho = math.sqrt(2) * r / 3.0
    prev = None
    for p in (4, 8, 12, 16):
        got = np.array([m2p(p2m(zs, q, c, r, p), c, r, z) for z in zt])
        err = rel(got, ex)
        assert err <= 2 * rho ** (p + 1) / (1 - rho), (p, err)
        if prev is not None:
            assert err < prev
        prev = err


def test_m2m_against_direct():
    """Four children's expansions moved to the parent centre give the parent's field."""
    rng = np.random.default_rng(2)
    cp, rp, p = 1.0 + 1.0j, 1.0, 16
    parts = []
    for dx in (-0.5, 0.5):
        for dy in (-0.5, 0.5):
            cc = cp + dx + 1j * dy
            zs, q = cluster(rng, cc, 0.5, 60)
            parts.append((zs, q, m2m(p2m(zs, q, cc, 0.5, p), cc, 0.5, cp, rp)))
    a = sum(x[2] for x in parts)
    zs = np.concatenate([x[0] for x in parts])
    q = np.concatenate([x[1] for x in parts])
    assert rel(a, p2m(zs, q, cp, rp, p)) < 1e-12      # M2M is exact (binomial identity)
    zt = cp + 5.0 * np.exp(2j * np.pi * rng.uniform(0, 1, 40))
    got = np.array([m2p(a, cp, rp, z) for z in zt])
    rho = math.sqrt(2) * rp / 5.0
    assert rel(got, direct(zt, zs, q)) <= 2 * rho ** (p + 1) / (1 - rho)


@pytest.mark.parametrize("dx,dy", [(2, 0), (0, -2), (3, 3), (-2, 3), (2, -1), (-3, -2)])
def test_m2l_offset_class_against_direct(dx, dy):
    """Source box at cell offset (dx, dy) from the target box, both half-width r:
    M2L of class w = 2 (dx + i dy), then L2P at points of the target box."""
    rng = np.random.default_rng(100 + 7 * dx + dy)
    r = 0.25
    ct = 0.1 + 0.7j
    cs = ct + 2 * r * (dx + 1j * dy)
    zs, q = cluster(rng, cs, r, 120)
    zt, _ = cluster(rng, ct, r, 40)
    ex = direct(zt, zs, q)
    w = 2 * (dx + 1j * dy)
    prev = None
    for p in (4, 8, 12, 16, 24):
        b = m2l_class(p2m(zs, q, cs, r, p), w)
        got = np.array([l2p(b, ct, r, z) for z in zt])
        err = rel(got, ex)
        ceiling = 2 * (1 + RHO_V) * RHO_V ** (p + 1) / (1 - RHO_V)
        assert err <= ceiling, (p, err, ceiling)
        if prev is not None and prev > 1e-13:
            assert err < prev
        prev = err


def test_m2l_class_matrix_does_not_depend_on_level():
    """The same cell offset at two levels: scaled coefficients give the same
    translated expansion, so one matrix per class serves every level."""
    rng = np.random.default_rng(4)
    p, dx, dy = 10, 3, -2
    for r in (1.0, 1 / 64):
        ct = 0.0
        cs = ct + 2 * r * (dx + 1j * dy)
        zs, q = cluster(rng, cs, r, 50)
        a = p2m(zs, q, cs, r, p)
        unscaled = np.zeros(p + 1, complex)
        au = a * r ** np.arange(p + 1)
        z0 = cs - ct
        for l in range(1, p + 1):
            unscaled[l] = -au[0] / (l * z0 ** l) + z0 ** (-l) * sum(
                (-1) ** k * au[k] * z0 ** (-k) * C(l + k - 1, k - 1) for k in range(1, p + 1))
        assert rel(m2l_class(a, 2 * (dx + 1j * dy)), unscaled * r ** np.arange(p + 1)) < 1e-12


def test_l2l_fold_is_exact():
    """The fold of an ancestor's incoming expansion into a leaf D levels finer
    is the binomial re-expansion: L2P of both agree to rounding."""
    rng = np.random.default_rng(5)
    p, rA = 12, 1.0
    cA = 0.0
    b = rng.normal(size=p + 1) + 1j * rng.normal(size=p + 1)
    b[0] = 0
    for D, (ix, iy) in ((1, (1, -1)), (3, (5, 3)), (5, (-31, 17))):
        rl = rA * 2.0 ** -D
        cl = cA + rl * ((ix) + 1j * (iy))           # centre of a descendant cell (odd offsets in units of rl)
        t = (cl - cA) / rA
        bl = l2l_fold(b, t, D)
        zt = cl + rl * (rng.uniform(-1, 1, 20) + 1j * rng.uniform(-1, 1, 20))
        a1 = np.array([l2p(b, cA, rA, z) for z in zt])
        a2 = np.array([l2p(bl, cl, rl, z) for z in zt])
        assert rel(a2, a1) < 1e-10, D


def test_p2l_against_direct():
    """Sources of an X-list leaf far from a box: P2L then L2P at the box's points."""
    rng = np.random.default_rng(6)
    r, c = 0.5, 0.0
    zs, q = cluster(rng, c + 4.0 + 1.0j, 0.25, 80)
    zt, _ = cluster(rng, c, r, 40)
    ex = direct(zt, zs, q)
    dmin = np.min(np.abs(zs - c))
    rho = math.sqrt(2) * r / dmin
    for p in (6, 12, 18):
        got = np.array([l2p(p2l(zs, q, c, r, p), c, r, z) for z in zt])
        assert rel(got, ex) <= 2 * rho ** (p + 1) / (1 - rho) + 1e-13, p


def test_field_gives_the_repulsion_of_o2():
    """kr m_i conj(E(z_i)) with q = m is kr m_i sum_j m_j (p_i - p_j) / |p_i - p_j|^2."""
    rng = np.random.default_rng(7)
    z = rng.normal(size=30) + 1j * rng.normal(size=30)
    m = rng.integers(1, 6, 30).astype(float)
    i = 4
    others = np.arange(30) != i
    E = np.sum(m[others] / (z[i] - z[others]))
    F = 2.5 * m[i] * np.conj(E)
    d = z[i] - z[others]
    Fx = 2.5 * m[i] * np.sum(m[others] * d.real / np.abs(d) ** 2)
    Fy = 2.5 * m[i] * np.sum(m[others] * d.imag / np.abs(d) ** 2)
    assert abs(F.real - Fx) < 1e-12 * abs(Fx) + 1e-12 and abs(F.imag - Fy) < 1e-12 * abs(Fy) + 1e-12
