"""Pins of the FP64 oracle's algebra against facts that do not come from the
oracle itself: the Hamilton table, the complex 2x2 matrix representation of the
quaternions, the dual-number block-matrix representation of dual quaternions,
Eq. quatsq, the magnitude of the appendix, and the complex Julia iteration of
Eq. julia as the special case of the 8-D iteration."""

import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(1234)
E = np.eye(4)  # 1, i, j, k


def cmat(q):
    """Quaternion a+bi+cj+dk as the complex 2x2 matrix [[a+bi, c+di], [-c+di, a-bi]]."""
    a, b, c, d = q
    return np.array([[a + 1j * b, c + 1j * d], [-c + 1j * d, a - 1j * b]])


def from_cmat(m):
    return np.array([m[0, 0].real, m[0, 0].imag, m[0, 1].real, m[0, 1].imag])


def dq_block(z):
    """Dual quaternion r + d eps as the 4x4 complex block matrix [[R, D], [0, R]];
    eps is the nilpotent block [[0, I], [0, 0]]."""
    R, D = cmat(z[:4]), cmat(z[4:])
    out = np.zeros((4, 4), complex)
    out[:2, :2] = R
    out[2:, 2:] = R
    out[:2, 2:] = D
    return out


def from_block(m):
    return np.concatenate([from_cmat(m[:2, :2]), from_cmat(m[:2, 2:])])


def close(a, b, rel=1e-12):
    a, b = np.asarray(a), np.asarray(b)
    scale = max(1.0, float(np.max(np.abs(b))))
    return float(np.max(np.abs(a - b))) <= rel * scale


def test_hamilton_table():
    one, i, j, k = E
    mul = oracle.quat_mul
    for u in (i, j, k):
        assert np.array_equal(mul(u, u), -one)
    assert np.array_equal(mul(i, j), k)
    assert np.array_equal(mul(j, k), i)
    assert np.array_equal(mul(k, i), j)
    assert np.array_equal(mul(j, i), -k)
    assert np.array_equal(mul(k, j), -i)
    assert np.array_equal(mul(i, k), -j)
    assert np.array_equal(mul(mul(i, j), k), -one)
    for u in E:
        assert np.array_equal(mul(one, u), u) and np.array_equal(mul(u, one), u)


def test_quat_mul_matches_complex_matrix_representation():
    for _ in range(2000):
        a, b = RNG.normal(size=4), RNG.normal(size=4)
        assert close(oracle.quat_mul(a, b), from_cmat(cmat(a) @ cmat(b)))


def test_quat_square_matches_eq_quatsq():
    # Eq. quatsq: q^2 = (x^2 - y^2 - z^2 - w^2, 2xy, 2xz, 2xw), real part first.
    for _ in range(2000):
        x, y, z, w = RNG.normal(size=4)
        want = [x * x - y * y - z * z - w * w, 2 * x * y, 2 * x * z, 2 * x * w]
        assert close(oracle.quat_mul([x, y, z, w], [x, y, z, w]), want)


def test_quat_norm_is_multiplicative_and_dot():
    for _ in range(500):
        a, b = RNG.normal(size=4), RNG.normal(size=4)
        p = oracle.quat_mul(a, b)
        assert abs(np.dot(p, p) - np.dot(a, a) * np.dot(b, b)) <= 1e-12 * np.dot(p, p)
        assert abs(oracle.quat_dot(a, b) - float(np.dot(a, b))) <= 1e-12 * (1 + abs(np.dot(a, b)))


def test_dq_mul_matches_block_matrix_representation():
    for _ in range(2000):
        a, b = RNG.normal(size=8), RNG.normal(size=8)
        assert close(oracle.dq_mul(a, b), from_block(dq_block(a) @ dq_block(b)))


def test_eps_squared_is_zero():
    eps = np.zeros(8)
    eps[4] = 1.0
    assert np.array_equal(oracle.dq_mul(eps, eps), np.zeros(8))
    # eps times any pure-dual dual quaternion vanishes too
    for _ in range(100):
        d = np.concatenate([np.zeros(4), RNG.normal(size=4)])
        assert np.array_equal(oracle.dq_mul(eps, d), np.zeros(8))


def test_dq_associative_and_distributive():
    for _ in range(1000):
        a, b, c = RNG.normal(size=(3, 8))
        lhs = oracle.dq_mul(oracle.dq_mul(a, b), c)
        rhs = oracle.dq_mul(a, oracle.dq_mul(b, c))
        assert close(lhs, rhs, 1e-12)
        lhs = oracle.dq_mul(a, oracle.dq_add(b, c))
        rhs = oracle.dq_add(oracle.dq_mul(a, b), oracle.dq_mul(a, c))
        assert close(lhs, rhs, 1e-12)


def test_dq_magnitude_is_dual_number():
    # zeta zeta* = |q_r|^2 + 2 (q_r . q_d) eps, a dual number (real scalars only)
    for _ in range(1000):
        z = RNG.normal(size=8)
        m = oracle.dq_magnitude(z)
        want = np.zeros(8)
        want[0] = np.dot(z[:4], z[:4])
        want[4] = 2.0 * np.dot(z[:4], z[4:])
        assert close(m, want, 1e-12)


def test_algebraic_square_expanded_form():
    # (r + d eps)^2 = r^2 + (r d + d r) eps; the cross products cancel in r d + d r,
    # leaving 2 (s_r s_d - v_r . v_d, s_r v_d + s_d v_r).
    for _ in range(2000):
        z = RNG.normal(size=8)
        r, d = z[:4], z[4:]
        want = np.concatenate([
            [r[0] ** 2 - r[1] ** 2 - r[2] ** 2 - r[3] ** 2, 2 * r[0] * r[1], 2 * r[0] * r[2],
             2 * r[0] * r[3]],
            2 * np.array([r[0] * d[0] - np.dot(r[1:], d[1:]), *(r[0] * d[1:] + d[0] * r[1:])]),
        ])
        assert close(oracle.dq_square(z, oracle.SQUARE_ALGEBRAIC), want)
        assert close(oracle.dq_square(z, oracle.SQUARE_ALGEBRAIC), from_block(dq_block(z) @ dq_block(z)))


def test_componentwise_square_is_eq_quatsq_on_both_halves():
    for _ in range(1000):
        z = RNG.normal(size=8)
        want = []
        for h in (z[:4], z[4:]):
            x, y, zz, w = h
            want += [x * x - y * y - zz * zz - w * w, 2 * x * y, 2 * x * zz, 2 * x * w]
        assert close(oracle.dq_square(z, oracle.SQUARE_PAPER_COMPONENTWISE), want)


def test_modulus_readings():
    for _ in range(200):
        z = RNG.normal(size=8)
        assert abs(oracle.modulus(z, oracle.MODULUS_EUCLID8) - np.dot(z, z)) <= 1e-12 * np.dot(z, z)
        assert abs(oracle.modulus(z, oracle.MODULUS_DUALNUM) - np.dot(z[:4], z[:4])) <= 1e-12 * np.dot(z, z)
        # DUALNUM is the modulus |a| of the dual number zeta zeta* (Introduction)
        assert abs(oracle.modulus(z, oracle.MODULUS_DUALNUM) - oracle.dq_magnitude(z)[0]) <= 1e-12 * np.dot(z, z)


@pytest.mark.parametrize("square_mode", [oracle.SQUARE_ALGEBRAIC, oracle.SQUARE_PAPER_COMPONENTWISE])
def test_real_part_is_quaternion_julia_iterate(square_mode):
    # The real half of the dual-quaternion iterate evolves as the quaternion Julia
    # map q <- q^2 + c_r (Eq. dqjulia), computed here with complex 2x2 matrices.
    for trial in range(200):
        # |z0| <= 0.6 and |c_r| <= 0.2 keep the quaternion orbit inside |q| <= 0.73
        z0 = RNG.uniform(-0.3, 0.3, 8)
        c = RNG.uniform(-0.1, 0.1, 8)
        n = int(RNG.integers(1, 33))
        Q, C = cmat(z0[:4]), cmat(c[:4])
        for _ in range(n):
            Q = Q @ Q + C
        zn = oracle.dq_julia(z0, c, n, square_mode)
        assert close(zn[:4], from_cmat(Q), 1e-12)
        assert close(oracle.quat_julia(z0[:4], c[:4], n), from_cmat(Q), 1e-12)


def test_dq_iterate_matches_block_matrix_iteration():
    for _ in range(300):
        z0 = RNG.uniform(-1, 1, 8)
        c = RNG.uniform(-0.8, 0.8, 8)
        n = int(RNG.integers(1, 6))
        Z, C = dq_block(z0), dq_block(c)
        for _ in range(n):
            Z = Z @ Z + C
        assert close(oracle.dq_julia(z0, c, n), from_block(Z), 1e-10)


@pytest.mark.parametrize("modulus_mode", [oracle.MODULUS_EUCLID8, oracle.MODULUS_DUALNUM])
def test_complex_special_case_escape_counts(modulus_mode):
    # Points (X, Y, 0, 0 | 0) with c = (a, b, 0, 0 | 0) stay in the complex
    # subalgebra: escape counts equal those of z <- z^2 + c (Eq. julia).
    for _ in range(3000):
        a, b = RNG.uniform(-1, 1, 2)
        x, y = RNG.uniform(-2, 2, 2)
        max_iter = int(RNG.integers(1, 40))
        z, c = complex(x, y), complex(a, b)
        want = 0
        for n in range(1, max_iter + 1):
            z = z * z + c
            if z.real * z.real + z.imag * z.imag > 16.0:
                want = n
                break
        got, _ = oracle.classify([x, y, 0, 0, 0, 0, 0, 0], [a, b, 0, 0, 0, 0, 0, 0], max_iter, 4.0,
                                 oracle.SQUARE_ALGEBRAIC, modulus_mode)
        assert got == want


def c0_escape_count(r, R, max_iter):
    """At c = 0 on a real-quaternion point of norm r, zeta_n = p^(2^n): escape at the
    first n >= 1 with r^(2^n) > R, or 0 (inside) if none up to max_iter."""
    if r <= 1.0:
        return 0
    n = max(1, int(np.floor(np.log2(np.log(R) / np.log(r)))) + 1)
    return n if n <= max_iter else 0


def test_c0_closed_form_escape_counts():
    checked = 0
    for _ in range(5000):
        r = float(np.exp(RNG.uniform(-3, 1)))
        dirn = RNG.normal(size=3)
        p = r * dirn / np.linalg.norm(dirn)
        max_iter = int(RNG.integers(1, 20))
        # skip points within rounding of an escape boundary r^(2^n) = R
        if r > 1.0:
            x = np.log2(np.log(4.0) / np.log(np.linalg.norm(p)))
            if abs(x - round(x)) < 1e-9:
                continue
        want = c0_escape_count(np.linalg.norm(p), 4.0, max_iter)
        got, _ = oracle.classify([p[0], p[1], p[2], 0, 0, 0, 0, 0], np.zeros(8), max_iter, 4.0)
        assert got == want, (p, max_iter)
        checked += 1
    assert checked > 4900


def test_escape_is_strict_and_first_update_is_tested():
    # m = R^2 exactly stays inside; zeta0 itself is never tested.
    # zeta0 = (2,0,0,0|0): zeta1 = 4 + c; with c = 0, m1 = 16 = R^2 -> not an escape.
    n, m = oracle.classify([2, 0, 0, 0, 0, 0, 0, 0], np.zeros(8), 1, 4.0)
    assert n == 0 and m == 16.0
    n, _ = oracle.classify([2, 0, 0, 0, 0, 0, 0, 0], np.zeros(8), 2, 4.0)
    assert n == 2
    # a starting point far outside still counts one update before escaping
    n, _ = oracle.classify([100, 0, 0, 0, 0, 0, 0, 0], np.zeros(8), 5, 4.0)
    assert n == 1
