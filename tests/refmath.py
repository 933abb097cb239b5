"""Reference mathematics for the tests: closed forms and quadratures of relativistic
phase space that do not come from the oracle or the CUDA path."""
import math
from fractions import Fraction

from scipy import integrate as spi

def minkowski2(p):
    """p[..., 4] -> E^2 - |p|^2."""
    return p[..., 0] ** 2 - (p[..., 1] ** 2 + p[..., 2] ** 2 + p[..., 3] ** 2)


def lam_exact(a, b, c):
    """Kallen lambda(a, b, c) = a^2 + b^2 + c^2 - 2ab - 2bc - 2ca in exact rationals."""
    a, b, c = Fraction(a), Fraction(b), Fraction(c)
    return a * a + b * b + c * c - 2 * a * b - 2 * b * c - 2 * c * a


def two_body_p(M, m1, m2):
    """sqrt(lambda(M^2, m1^2, m2^2)) / (2 M), lambda evaluated exactly."""
    lam = lam_exact(Fraction(M) ** 2, Fraction(m1) ** 2, Fraction(m2) ** 2)
    return math.sqrt(max(float(lam), 0.0)) / (2.0 * M)


def massless_volume(n, M):
    """R_n = (pi/2)^(n-1) M^(2n-4) / ((n-1)! (n-2)!)  (massless n-body phase space)."""
    return (math.pi / 2) ** (n - 1) * M ** (2 * n - 4) / (math.factorial(n - 1) * math.factorial(n - 2))


def R2(M, a, b):
    """Two-body volume Int d3p1/(2E1) d3p2/(2E2) delta4 = pi p* / M."""
    if M <= a + b:
        return 0.0
    return math.pi * two_body_p(M, a, b) / M


def R_recursive(M, masses, epsrel=1e-8):
    """R_n(M) = Int ds R_2(M; sqrt(s), m_n) R_{n-1}(sqrt(s)) by nested adaptive quadrature."""
    n = len(masses)
    if n == 2:
        return R2(M, masses[0], masses[1])
    lo = sum(masses[:-1]) ** 2
    hi = (M - masses[-1]) ** 2

    def integrand(s):
        ms = math.sqrt(s)
        return R2(M, ms, masses[-1]) * R_recursive(ms, masses[:-1], epsrel)

    val, _ = spi.quad(integrand, lo, hi, epsabs=0, epsrel=epsrel, limit=100)
    return val


def dalitz_s23_range(M, m1, m2, m3, s12):
    m12 = math.sqrt(s12)
    E2 = (s12 - m1 * m1 + m2 * m2) / (2 * m12)
    E3 = (M * M - s12 - m3 * m3) / (2 * m12)
    q2 = math.sqrt(max(E2 * E2 - m2 * m2, 0.0))
    q3 = math.sqrt(max(E3 * E3 - m3 * m3, 0.0))
    return (E2 + E3) ** 2 - (q2 + q3) ** 2, (E2 + E3) ** 2 - (q2 - q3) ** 2


def R3_quad(M, m):
    """R_3 = pi^2 / (4 M^2) * Dalitz-plot area."""
    m1, m2, m3 = m

    def width(s12):
        lo, hi = dalitz_s23_range(M, m1, m2, m3, s12)
        return hi - lo

    area, _ = spi.quad(width, (m1 + m2) ** 2, (M - m3) ** 2, epsabs=0, epsrel=1e-12, limit=200)
    return math.pi ** 2 / (4 * M * M) * area



def dalitz_me_integral_quad(M, masses, params):
    """Int |ME|^2 dR_3 = pi^2/(4M^2) Int Int |ME|^2 ds12 ds23 by 2-D adaptive quadrature with
    the resonance poles as break points; ME = BW(s12; a) + c BW(s23; b), c = |c| e^{i arg c}."""
    m1, m2, m3 = masses
    m0a, Ga, m0b, Gb, cm, ca = params
    c = cm * complex(math.cos(ca), math.sin(ca))

    def me2(s12, s23):
        amp = 1.0 / complex(m0a * m0a - s12, -m0a * Ga) + c / complex(m0b * m0b - s23, -m0b * Gb)
        return abs(amp) ** 2

    def inner(s12):
        lo, hi = dalitz_s23_range(M, m1, m2, m3, s12)
        pts = [m0b * m0b] if lo < m0b * m0b < hi else None
        v, _ = spi.quad(lambda s23: me2(s12, s23), lo, hi, points=pts, epsabs=0,
                        epsrel=1e-10, limit=400)
        return v

    lo12, hi12 = (m1 + m2) ** 2, (M - m3) ** 2
    pts = [m0a * m0a] if lo12 < m0a * m0a < hi12 else None
    outer, _ = spi.quad(inner, lo12, hi12, points=pts, epsabs=0, epsrel=1e-9, limit=400)
    return math.pi ** 2 / (4 * M * M) * outer, me2
