"""The algebra behind the FP32 kernels' WENO5 arithmetic, checked in FP64 against the
textbook WENO5-JS face value (Jiang & Shu 1996, the scheme the paper cites) and against
central differences: the weights depend only on ratios of (eps + beta_k)^2, so scaling the
smoothness indicators and eps by 12/13 and the linear weights by 10, with numerator and
denominator factored around A1, gives the same face value; the derivative of that value with
respect to the five stencil values, written on first differences with the factor 2 of
d beta'/dv folded into the sensitivity factors, matches finite differences.  (The CUDA
kernels are checked against the oracle by the GPU tests; this pins the restatement.)"""
import numpy as np


def textbook(v, eps=1e-6):
    a, b, c, d, e = v
    q = [(2 * a - 7 * b + 11 * c) / 6, (-b + 5 * c + 2 * d) / 6, (2 * c + 5 * d - e) / 6]
    beta = [13 / 12 * (a - 2 * b + c) ** 2 + 0.25 * (a - 4 * b + 3 * c) ** 2,
            13 / 12 * (b - 2 * c + d) ** 2 + 0.25 * (b - d) ** 2,
            13 / 12 * (c - 2 * d + e) ** 2 + 0.25 * (3 * c - 4 * d + e) ** 2]
    al = [dk / (eps + bk) ** 2 for dk, bk in zip((0.1, 0.6, 0.3), beta)]
    return sum(x * y for x, y in zip(al, q)) / sum(al)


def factored(v, eps=1e-6):
    """The forward kernels' form: first differences, beta and eps scaled by 12/13,
    q-weights A1 A2 : 6 A0 A2 : 3 A0 A1 with one division."""
    a, b, c, d, e = v
    d1, d2, d3, d4 = b - a, c - b, d - c, e - d
    s = (d2 - d1, d3 - d2, d4 - d3)
    t = (3 * d2 - d1, d2 + d3, -3 * d3 + d4)
    k, ep = 3 / 13, eps * 12 / 13
    A0, A1, A2 = ((sk * sk + k * tk * tk + ep) ** 2 for sk, tk in zip(s, t))
    r0, r1, r2 = 5 * d2 - 2 * d1, 2 * d3 + d2, 4 * d3 - d4
    a02x6 = 6 * A0 * A2
    num = A1 * (3 * A0 * r2 + A2 * r0) + a02x6 * r1
    den = A1 * (3 * A0 + A2) + a02x6
    return c + num / den / 6


def value_and_grad(v, eps=1e-6):
    """The adjoint kernels' form of the value and its five partial derivatives."""
    a, b, c, d, e = v
    d1, d2, d3, d4 = b - a, c - b, d - c, e - d
    dq = (5 / 6 * d2 - d1 / 3, d3 / 3 + d2 / 6, 2 / 3 * d3 - d4 / 6)
    s0, s1, s2 = d2 - d1, d3 - d2, d4 - d3
    t0, t1, t2 = 3 * d2 - d1, d2 + d3, -3 * d3 + d4
    k, ep = 3 / 13, eps * 12 / 13
    kt0, kt1, kt2 = k * t0, k * t1, k * t2
    i0, i1, i2 = 1 / (s0 * s0 + kt0 * t0 + ep), 1 / (s1 * s1 + kt1 * t1 + ep), 1 / (s2 * s2 + kt2 * t2 + ep)
    a0, a1, a2 = 0.1 * i0 * i0, 0.6 * i1 * i1, 0.3 * i2 * i2
    inv = 1 / (a0 + a1 + a2)
    w0, w1, w2 = a0 * inv, a1 * inv, a2 * inv
    dval = w0 * dq[0] + w1 * dq[1] + w2 * dq[2]
    r0, r1, r2 = (-4 * (dq[m] - dval) * (w * i) for m, w, i in ((0, w0, i0), (1, w1, i1), (2, w2, i2)))
    dv = np.array([w0 / 3 + r0 * (s0 + kt0),
                   -7 / 6 * w0 - w1 / 6 + r0 * (-2 * s0 - 4 * kt0) + r1 * (s1 - kt1),
                   11 / 6 * w0 + 5 / 6 * w1 + w2 / 3 + r0 * (s0 + 3 * kt0) + r1 * (-2 * s1) + r2 * (s2 + 3 * kt2),
                   w1 / 3 + 5 / 6 * w2 + r1 * (s1 + kt1) + r2 * (-2 * s2 - 4 * kt2),
                   -w2 / 6 + r2 * (s2 + kt2)])
    return c + dval, dv


def _stencils(count, seed):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        yield rng.normal(size=5) * 10.0 ** rng.uniform(-3, 0)
    yield np.array([0.0, 0.0, 1.0, 1.0, 1.0])   # a jump
    yield np.array([1.0, 2.0, 3.0, 4.0, 5.0])   # linear data


def test_factored_face_value_is_the_textbook_value():
    for v in _stencils(2000, 0):
        ref = textbook(v)
        assert abs(factored(v) - ref) <= 1e-13 * max(1.0, abs(ref))
        assert abs(value_and_grad(v)[0] - ref) <= 1e-13 * max(1.0, abs(ref))


def test_adjoint_derivative_matches_central_differences():
    for v in _stencils(500, 1):
        _, dv = value_and_grad(v)
        h = 1e-6 * max(1e-3, np.abs(v).max())
        fd = np.array([(value_and_grad(v + h * ej)[0] - value_and_grad(v - h * ej)[0]) / (2 * h)
                       for ej in np.eye(5)])
        assert np.abs(fd - dv).max() <= 1e-7 * max(1.0, np.abs(dv).max())
