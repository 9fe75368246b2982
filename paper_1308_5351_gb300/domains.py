"""Seeded synthetic boundaries and right-hand sides (input generation only).

This module produces the *inputs* of the method: the composite boundary
parametrisation eta(t) with its derivatives on the node grid, the coefficient
function A(t) with A'(t), and right-hand sides gamma.  It contains none of the
method's arithmetic (no kernel, no quadrature, no solve), so both the dense
CPU oracle and the CUDA library are fed from here.

Conventions (paper Sec. 2.1, 2.4):
  * G has m+1 boundary components Gamma_0..Gamma_m, each a 2*pi-periodic curve
    eta_j(t); G lies to the left of Gamma.  Bounded G: Gamma_0 is the outer curve
    (counter-clockwise) and the holes are clockwise.  Unbounded G: every
    component is clockwise.
  * Nodes: t_{kn+p} = (p-1) 2 pi / n, component-major (Eq. ti-skp), n even.
  * A(t) = exp(i(pi/2 - theta_j)) (eta(t) - alpha) for bounded G and
    exp(i(pi/2 - theta_j)) for unbounded G (Eq. A), theta piecewise constant
    (Eq. thet).
  * Piecewise-smooth components are parametrised on the graded mesh of Sec. 6:
    eta_j = zeta_j o delta_j (Eq. zet-et) with delta_j built from omega
    (Eq. omega, omega-v, delta_j).

All arrays are numpy complex128 of length (m+1) n.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence

import numpy as np

TWO_PI = 2.0 * math.pi


# --------------------------------------------------------------------------
# Curves: each returns (z, z', z'') at parameter values t (numpy arrays)
# --------------------------------------------------------------------------

class Curve:
    """A 2*pi-periodic parametrised closed curve."""

    corners = 0  # number of corner points (graded mesh), 0 if smooth

    def eval(self, t: np.ndarray):  # pragma: no cover - interface
        raise NotImplementedError

    def bbox_radius(self) -> float:  # pragma: no cover - interface
        raise NotImplementedError


@dataclasses.dataclass
class Circle(Curve):
    centre: complex
    radius: float
    ccw: bool = False

    def eval(self, t):
        s = 1.0 if self.ccw else -1.0
        e = np.exp(1j * s * t)
        z = self.centre + self.radius * e
        zp = 1j * s * self.radius * e
        zpp = -self.radius * e
        return z, zp, zpp

    def bbox_radius(self):
        return self.radius


@dataclasses.dataclass
class Ellipse(Curve):
    """centre + exp(i phi) (a cos t + i s b sin t), s = +1 ccw, -1 cw."""
    centre: complex
    a: float
    b: float
    phi: float = 0.0
    ccw: bool = False

    def eval(self, t):
        s = 1.0 if self.ccw else -1.0
        rot = np.exp(1j * self.phi)
        z = self.centre + rot * (self.a * np.cos(t) + 1j * s * self.b * np.sin(t))
        zp = rot * (-self.a * np.sin(t) + 1j * s * self.b * np.cos(t))
        zpp = rot * (-self.a * np.cos(t) - 1j * s * self.b * np.sin(t))
        return z, zp, zpp

    def bbox_radius(self):
        return max(self.a, self.b)


@dataclasses.dataclass
class Star(Curve):
    """centre + r(th) e^{i th}, th = +-t, r(th) = r0 (1 + sum a_k cos k th + b_k sin k th)."""
    centre: complex
    r0: float
    ak: np.ndarray
    bk: np.ndarray
    ccw: bool = False

    def eval(self, t):
        s = 1.0 if self.ccw else -1.0
        th = s * t
        k = np.arange(1, len(self.ak) + 1)[:, None]
        c = np.cos(k * th[None, :])
        sn = np.sin(k * th[None, :])
        a = np.asarray(self.ak)[:, None]
        b = np.asarray(self.bk)[:, None]
        r = self.r0 * (1.0 + np.sum(a * c + b * sn, axis=0))
        dr = self.r0 * np.sum(k * (-a * sn + b * c), axis=0)          # d r / d th
        ddr = self.r0 * np.sum(-(k ** 2) * (a * c + b * sn), axis=0)  # d2 r / d th2
        e = np.exp(1j * th)
        z = self.centre + r * e
        dz_dth = (dr + 1j * r) * e
        d2z_dth2 = (ddr + 2j * dr - r) * e
        return z, s * dz_dth, d2z_dth2  # s^2 = 1

    def bbox_radius(self):
        return self.r0 * (1.0 + float(np.sum(np.abs(self.ak) + np.abs(self.bk))))


# ---- graded mesh of Sec. 6 -------------------------------------------------

def _v(u, p):
    """v(t) of Eq. (omega-v) and its first two derivatives."""
    c1 = 1.0 / p - 0.5
    w = (math.pi - u) / math.pi
    v = c1 * w ** 3 + (u - math.pi) / (p * math.pi) + 0.5
    dv = -3.0 * c1 * w ** 2 / math.pi + 1.0 / (p * math.pi)
    ddv = 6.0 * c1 * w / math.pi ** 2
    return v, dv, ddv


def grading_omega(u: np.ndarray, p: int):
    """omega(u) of Eq. (omega) on [0, 2 pi] with omega' and omega''.

    omega = 2 pi P / (P + Q), P = v(u)^p, Q = v(2 pi - u)^p.
    """
    a, da, dda = _v(u, p)
    b, db, ddb = _v(TWO_PI - u, p)
    db = -db  # d/du of v(2 pi - u)
    P = a ** p
    Q = b ** p
    dP = p * a ** (p - 1) * da
    dQ = p * b ** (p - 1) * db
    ddP = p * (p - 1) * a ** (p - 2) * da ** 2 + p * a ** (p - 1) * dda
    ddQ = p * (p - 1) * b ** (p - 2) * db ** 2 + p * b ** (p - 1) * ddb
    W = P + Q
    U = dP * Q - P * dQ
    dU = ddP * Q - P * ddQ
    s = P / W
    ds = U / W ** 2
    dds = (dU * W - 2.0 * U * (dP + dQ)) / W ** 3
    return TWO_PI * s, TWO_PI * ds, TWO_PI * dds


def grading_delta(t: np.ndarray, pj: int, p: int):
    """delta_j(t) of Eq. (delta_j) with pj corners at c_k = (k-1) 2 pi / pj.

    Returns (delta, delta', delta'').
    """
    t = np.mod(np.asarray(t, dtype=np.float64), TWO_PI)
    h = TWO_PI / pj
    k = np.minimum(np.floor(t / h), pj - 1)
    ck = k * h
    om, dom, ddom = grading_omega(pj * (t - ck), p)
    return om / pj + ck, dom, ddom * pj


@dataclasses.dataclass
class GradedPolygon(Curve):
    """Polygon zeta_j (piecewise linear, corners at c_k = (k-1) 2 pi/pj) on the
    graded mesh: eta = zeta o delta (Eq. zet-et).  Vertices listed in the
    traversal order (ccw or cw is the caller's choice)."""
    vertices: Sequence[complex]
    p: int = 3

    def __post_init__(self):
        self.vertices = [complex(v) for v in self.vertices]
        self.corners = len(self.vertices)
        self.centre = complex(np.mean(self.vertices))

    def eval(self, t):
        pj = len(self.vertices)
        V = np.asarray(self.vertices, dtype=np.complex128)
        t = np.mod(np.asarray(t, dtype=np.float64), TWO_PI)
        hstep = TWO_PI / pj
        k = np.minimum(np.floor(t / hstep), pj - 1).astype(np.int64)
        ck = k * hstep
        om, dom, ddom = grading_omega(pj * (t - ck), self.p)
        edge = V[(k + 1) % pj] - V[k]
        frac = om / TWO_PI
        z = V[k] + edge * frac
        zp = edge * dom * pj / TWO_PI
        zpp = edge * ddom * pj * pj / TWO_PI
        return z, zp, zpp

    def bbox_radius(self):
        return float(np.max(np.abs(np.asarray(self.vertices) - self.centre)))


def square(centre: complex, half: float, ccw: bool, rot: float = 0.0, p: int = 3):
    """Axis-aligned (then rotated) square with graded corners."""
    base = [1 + 1j, -1 + 1j, -1 - 1j, 1 - 1j] if ccw else [1 + 1j, 1 - 1j, -1 - 1j, -1 + 1j]
    r = np.exp(1j * rot)
    return GradedPolygon([centre + half * r * v for v in base], p=p)


# --------------------------------------------------------------------------
# Domain: discretised boundary + coefficient A
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Domain:
    """Discretised (m+1)-connected domain.

    et, etp, etpp : eta, eta', eta'' at the (m+1) n nodes (component-major)
    A, Ap         : A(t), A'(t) of Eq. (A) at the nodes
    theta         : piecewise constant theta_j (length m+1)
    alpha         : the fixed point alpha of bounded G (None if unbounded)
    holes         : one interior point per hole (outside G), used for poles of
                    manufactured solutions and for log|eta - alpha_k| RHS
    """
    n: int
    bounded: bool
    curves: List[Curve]
    theta: np.ndarray
    alpha: Optional[complex]
    holes: List[complex]
    et: np.ndarray
    etp: np.ndarray
    etpp: np.ndarray
    A: np.ndarray
    Ap: np.ndarray

    @property
    def m1(self) -> int:
        return len(self.curves)

    @property
    def N(self) -> int:
        return self.m1 * self.n

    @property
    def c(self) -> int:
        """c of Eq. (c): +1 bounded, -1 unbounded."""
        return 1 if self.bounded else -1

    def component_of_node(self) -> np.ndarray:
        return np.repeat(np.arange(self.m1), self.n)


def nodes(n: int) -> np.ndarray:
    """s_{k,p} = (p-1) 2 pi / n, p = 1..n (Sec. 2.4)."""
    return np.arange(n, dtype=np.float64) * (TWO_PI / n)


def build_domain(curves: Sequence[Curve], n: int, bounded: bool,
                 theta: Optional[Sequence[float]] = None,
                 alpha: Optional[complex] = None,
                 holes: Optional[Sequence[complex]] = None) -> Domain:
    """Discretise the curves at n nodes each and form A, A' (Eq. A)."""
    if n % 2 != 0 or n < 4:
        raise ValueError("n must be even and >= 4")
    m1 = len(curves)
    if theta is None:
        theta = np.full(m1, math.pi / 2)
    theta = np.asarray(theta, dtype=np.float64)
    if theta.shape != (m1,):
        raise ValueError("theta must have one value per component")
    if bounded and alpha is None:
        raise ValueError("bounded G needs alpha")
    t = nodes(n)
    zs, zps, zpps = [], [], []
    for cv in curves:
        z, zp, zpp = cv.eval(t)
        zs.append(np.broadcast_to(z, t.shape))
        zps.append(np.broadcast_to(zp, t.shape))
        zpps.append(np.broadcast_to(zpp, t.shape))
    et = np.concatenate(zs).astype(np.complex128)
    etp = np.concatenate(zps).astype(np.complex128)
    etpp = np.concatenate(zpps).astype(np.complex128)
    rot = np.repeat(np.exp(1j * (math.pi / 2 - theta)), n)
    if bounded:
        A = rot * (et - alpha)
        Ap = rot * etp
    else:
        A = rot.astype(np.complex128)
        Ap = np.zeros_like(et)
    if holes is None:
        hs = [cv.centre for cv in curves]
        if bounded:
            hs = [complex(alpha)] + hs[1:]  # component 0 is the outer curve
        holes = hs
    return Domain(n=n, bounded=bounded, curves=list(curves), theta=theta,
                  alpha=None if alpha is None else complex(alpha),
                  holes=[complex(h) for h in holes], et=et, etp=etp,
                  etpp=etpp, A=A, Ap=Ap)


# --------------------------------------------------------------------------
# Right-hand sides
# --------------------------------------------------------------------------

def gamma_log(dom: Domain, a: complex) -> np.ndarray:
    """gamma(t) = log|eta(t) - a|."""
    return np.log(np.abs(dom.et - a))


def manufactured(dom: Domain, f: Callable[[np.ndarray], np.ndarray]):
    """gamma = Re[A f(eta)], exact mu = Im[A f(eta)], exact h = 0 (Sec. 7, Ex. 1)."""
    Af = dom.A * f(dom.et)
    return Af.real.copy(), Af.imag.copy()


def f_bounded_ex1(z):
    """f(z) = sin z + 1/(z-2) (Eq. ex-fb)."""
    return np.sin(z) + 1.0 / (z - 2.0)


def f_unbounded_ex1(z):
    """f(z) = 1/z - sin(1/z) (Eq. ex-fu); analytic where 0 lies in a hole."""
    return 1.0 / z - np.sin(1.0 / z)


def f_poles(poles: Sequence[complex], weights: Sequence[complex]):
    """f(z) = sum_k w_k / (z - z_k): analytic in G when every pole is in a hole,
    with f(inf) = 0."""
    P = np.asarray(poles, dtype=np.complex128)
    W = np.asarray(weights, dtype=np.complex128)

    def f(z):
        z = np.asarray(z)
        return np.sum(W[:, None] / (z[None, :] - P[:, None]), axis=0)
    return f


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------

def disk(n: int, alpha: complex = 0.3 + 0.2j) -> Domain:
    """Unit disk, A = eta - alpha."""
    return build_domain([Circle(0j, 1.0, ccw=True)], n, bounded=True, alpha=alpha)


def annulus(n: int, r: float = 0.5, alpha: complex = 0.75 + 0j) -> Domain:
    """Annulus r < |z| < 1, A = eta - alpha with alpha in G."""
    return build_domain([Circle(0j, 1.0, ccw=True), Circle(0j, r, ccw=False)],
                        n, bounded=True, alpha=alpha)


def three_circles(n: int = 256, alpha: complex = 0.05j,
                  theta: Optional[Sequence[float]] = None) -> Domain:
    """Bounded connectivity-3 domain: unit circle, holes of radius 0.2 at +-0.45.

    A = eta - alpha (theta = pi/2), alpha = 0.05 i (the point of gamma)."""
    curves = [Circle(0j, 1.0, ccw=True), Circle(0.45 + 0j, 0.2), Circle(-0.45 + 0j, 0.2)]
    return build_domain(curves, n, bounded=True, alpha=alpha, theta=theta)


def ex2_circles(eps: float, n: int, theta: Optional[Sequence[float]] = None,
                alpha: complex = 0j) -> Domain:
    """Bounded 5-circle domain of Example 2 (radius and centres as printed)."""
    s = 2.0 + 2.0 * math.sqrt(2.0)
    rho = (2.0 - eps * s) / s
    c = (2.0 - eps) / s
    curves = [Circle(0j, 1.0, ccw=True)]
    for sx, sy in ((1, 1), (-1, 1), (-1, -1), (1, -1)):
        curves.append(Circle(complex(sx * c, sy * c), rho))
    return build_domain(curves, n, bounded=True, alpha=alpha, theta=theta)


def ex4_circles(eps: float, n: int, theta: Optional[Sequence[float]] = None) -> Domain:
    """Unbounded 5-circle domain of Example 4 (gaps exactly eps)."""
    curves = [Circle(0j, math.sqrt(2.0) - 1.0 - eps / 2.0)]
    for sx, sy in ((1, 1), (-1, 1), (-1, -1), (1, -1)):
        curves.append(Circle(complex(sx, sy), 1.0 - eps / 2.0))
    return build_domain(curves, n, bounded=False, theta=theta)


def _polyline(cv: Curve, npts: int = 4096) -> np.ndarray:
    z, _, _ = cv.eval(np.linspace(0.0, TWO_PI, npts, endpoint=False))
    return np.asarray(z)


def _min_gap(za: np.ndarray, zb: np.ndarray) -> float:
    d = np.abs(za[:, None] - zb[None, :])
    return float(d.min())


def random_ellipses(rng: np.random.Generator, count: int, box: float,
                    axes=(0.1, 0.4), min_gap: float = 0.05,
                    poly_pts: int = 512, max_tries: int = 200000) -> List[Curve]:
    """Rejection-sample non-overlapping clockwise ellipses with centres in
    [-box, box]^2, semi-axes U[axes], rotation U[0, pi); the gap between any
    two is at least min_gap (checked on polylines)."""
    out: List[Curve] = []
    polys: List[np.ndarray] = []
    tries = 0
    while len(out) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place ellipses")
        c = complex(rng.uniform(-box, box), rng.uniform(-box, box))
        a, b = rng.uniform(axes[0], axes[1], size=2)
        phi = rng.uniform(0.0, math.pi)
        cand = Ellipse(c, float(a), float(b), float(phi), ccw=False)
        R = max(a, b)
        ok = True
        for e, pl in zip(out, polys):
            dc = abs(e.centre - c)
            if dc > R + e.bbox_radius() + min_gap:
                continue
            if dc < max(R, e.bbox_radius()):
                ok = False
                break
            zc = _polyline(cand, poly_pts)
            # point-in-ellipse rejects containment; polyline distance gap
            if _min_gap(zc, pl) < min_gap:
                ok = False
                break
        if ok:
            out.append(cand)
            polys.append(_polyline(cand, poly_pts))
    return out


def ellipses64(seed: int = 2, n: int = 1024, count: int = 64) -> Domain:
    """Unbounded domain exterior to `count` ellipses: centres U[-4,4]^2,
    semi-axes U[0.1,0.4], rotation U[0,pi), min gap >= 0.05; A = 1."""
    rng = np.random.default_rng(seed)
    curves = random_ellipses(rng, count, 4.0)
    return build_domain(curves, n, bounded=False)


def close_curves(seed: int = 3, n: int = 512, grid: int = 32, cell: float = 0.07,
                 squares: int = 32, close_frac: float = 0.1) -> Domain:
    """High-connectivity unbounded domain with close boundaries.

    grid x grid cells of size `cell`; in each a circle or ellipse of radius
    U[0.01, 0.03] (half are ellipses with semi-axes r and r U[0.5,1], random
    rotation), `squares` of them replaced by graded squares (p = 3).  About
    close_frac of horizontally adjacent circle pairs are moved together to a
    gap of 10^U(-3,0) times the smaller radius.
    """
    rng = np.random.default_rng(seed)
    total = grid * grid
    kinds = np.where(rng.uniform(size=total) < 0.5, 1, 0)  # 1 ellipse, 0 circle
    sq_idx = rng.choice(total, size=squares, replace=False)
    kinds[sq_idx] = 2
    radii = rng.uniform(0.01, 0.03, size=total)
    jit = rng.uniform(-0.0025, 0.0025, size=(total, 2))
    centres = np.empty(total, dtype=np.complex128)
    for gy in range(grid):
        for gx in range(grid):
            k = gy * grid + gx
            centres[k] = complex((gx - (grid - 1) / 2) * cell + jit[k, 0],
                                 (gy - (grid - 1) / 2) * cell + jit[k, 1])
    # move some circle pairs close together (exact gap for circles)
    for gy in range(grid):
        for gx in range(0, grid - 1, 2):
            k, k2 = gy * grid + gx, gy * grid + gx + 1
            if kinds[k] == 0 and kinds[k2] == 0 and rng.uniform() < 2 * close_frac:
                g = 10.0 ** rng.uniform(-3.0, 0.0) * min(radii[k], radii[k2])
                # place k2 on the ray from k through k2 at distance r+r2+g
                d = centres[k2] - centres[k]
                d /= abs(d)
                centres[k2] = centres[k] + d * (radii[k] + radii[k2] + g)
    curves: List[Curve] = []
    for k in range(total):
        r = float(radii[k])
        if kinds[k] == 0:
            curves.append(Circle(complex(centres[k]), r, ccw=False))
        elif kinds[k] == 1:
            curves.append(Ellipse(complex(centres[k]), r, r * float(rng.uniform(0.5, 1.0)),
                                  float(rng.uniform(0.0, math.pi)), ccw=False))
        else:
            curves.append(square(complex(centres[k]), r / math.sqrt(2.0), ccw=False,
                                 rot=float(rng.uniform(0.0, math.pi / 2))))
    return build_domain(curves, n, bounded=False)


def batch_domains(seed: int = 4, count: int = 256, conn=(2, 64),
                  ns=(128, 256, 512, 1024)) -> List[Domain]:
    """Independent unbounded domains with connectivity U{conn} and n U{ns}:
    ellipses placed like `ellipses64`, box scaled to the connectivity."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m1 = int(rng.integers(conn[0], conn[1] + 1))
        n = int(rng.choice(ns))
        box = 4.0 * math.sqrt(m1 / 64.0) + 0.5
        curves = random_ellipses(rng, m1, box)
        out.append(build_domain(curves, n, bounded=False))
    return out


def stars_and_polygons(seed: int = 5, n: int = 2048, kmax: int = 64,
                       r0: float = 0.3, spacing: float = 1.0) -> Domain:
    """Unbounded domain: 16 star-shaped curves r0 (1 + sum_{k<=kmax} a_k cos k th
    + b_k sin k th), a_k, b_k ~ N(0, (0.05/k)^2), and 4 graded polygons
    (2 squares, 2 triangles), on a 5 x 4 grid of spacing 1."""
    rng = np.random.default_rng(seed)
    curves: List[Curve] = []
    slots = [complex(x * spacing, y * spacing) for y in range(4) for x in range(5)]
    poly_slots = {3, 6, 13, 16}
    for s, c in enumerate(slots):
        if s in poly_slots:
            if len(curves) % 2 == 0:
                curves.append(square(c, r0 * 0.8, ccw=False, rot=float(rng.uniform(0, 1))))
            else:
                ang = float(rng.uniform(0, TWO_PI))
                verts = [c + r0 * np.exp(1j * (ang - TWO_PI * q / 3)) for q in range(3)]
                curves.append(GradedPolygon(verts, p=3))
        else:
            k = np.arange(1, kmax + 1)
            ak = rng.normal(0.0, 0.05 / k)
            bk = rng.normal(0.0, 0.05 / k)
            curves.append(Star(c, r0, ak, bk, ccw=False))
    return build_domain(curves, n, bounded=False)


def config_domain(idx: int) -> Domain:
    """The five workload configurations (1-based index), at their full sizes."""
    if idx == 1:
        return three_circles(256)
    if idx == 2:
        return ellipses64(2, 1024)
    if idx == 3:
        return close_curves(3, 512)
    if idx == 5:
        return stars_and_polygons(5, 2048)
    raise ValueError("config 4 is a list of domains: use batch_domains()")


def pack_complex(z: np.ndarray) -> np.ndarray:
    """complex128 (N,) -> float64 (N, 2) interleaved (re, im) as the C ABI expects."""
    z = np.ascontiguousarray(z, dtype=np.complex128)
    return z.view(np.float64).reshape(-1, 2)
