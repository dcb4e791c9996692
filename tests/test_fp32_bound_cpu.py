"""CPU check of the FP32 filter's error bounds (the diameter engine's header
states them; Sec. 2's diameter is the FP64 maximum, the FP32 pass only
selects candidates).  The kernels' FP32 operations are emulated exactly here:
numpy float32 arithmetic rounds each operation to nearest, and a fused
multiply-add is evaluated in exact rational arithmetic and rounded once.

Positions are P = fl32((u - c) s) with u the index position of a vertex (a
half-integer along its edge's axis), c the grid centre and s the spacing;
R is the half diagonal of the padded grid.  Checked:
  expansion form  g = fl(n_a + fma(-2P_ax, P_bx, fma(-2P_ay, P_by, fma(-2P_az, P_bz, n_b))))
                  |g - d2| <= 4.1u R sqrt(d2) + 20.2u R^2
  difference form f = fma(dz, dz, fma(dy, dy, fl(dx dx))), d = fl(P_a - P_b)
                  |f - d2| <= 5.1u d2 + 4.1u R sqrt(d2) + 4.1u^2 R^2
and that the threshold T(F) built from the doubled coefficients keeps every
pair attaining the exact maximum for the largest F any pair can produce."""
from fractions import Fraction

import numpy as np
import pytest

U = 2.0 ** -24
GRIDS = [((512, 512, 256), (0.7, 0.7, 2.5)), ((160, 160, 160), (1.0, 1.0, 1.0)),
         ((192, 100, 40), (0.8, 0.8, 3.0)), ((64, 48, 96), (0.5, 0.5, 1.0))]


def round32(q):
    """Fraction -> nearest float32, ties to even."""
    x = np.float32(float(q))
    cands = [x, np.nextafter(x, np.float32(np.inf)), np.nextafter(x, np.float32(-np.inf))]
    return min(cands, key=lambda y: (abs(Fraction(float(y)) - q), int(np.float32(y).view(np.uint32)) & 1))


def fma32(a, b, c):
    return round32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def entry(u, dims, sp):
    """FP32 position and norm of one vertex, as the sort kernel stores them."""
    c = [0.5 * (n - 1) for n in dims]
    P = [np.float32((u[k] - c[k]) * sp[k]) for k in range(3)]
    n = np.float32(np.float32(P[0] * P[0]) + np.float32(P[1] * P[1]))
    n = np.float32(n + np.float32(P[2] * P[2]))
    return P, n


def g_expansion(ea, eb):
    (Pa, na), (Pb, nb) = ea, eb
    a2 = [np.float32(-2.0) * Pa[k] for k in range(3)]  # exact
    h = fma32(a2[2], Pb[2], nb)
    h = fma32(a2[1], Pb[1], h)
    h = fma32(a2[0], Pb[0], h)
    return np.float32(na + h)


def f_difference(ea, eb):
    Pa, Pb = ea[0], eb[0]
    d = [np.float32(Pa[k] - Pb[k]) for k in range(3)]
    f = np.float32(d[0] * d[0])
    f = fma32(d[1], d[1], f)
    return fma32(d[2], d[2], f)


def exact_d2(ua, ub, sp):
    return sum((Fraction(ua[k]) - Fraction(ub[k])) ** 2 * Fraction(sp[k]) ** 2 for k in range(3))


def radius2(dims, sp):
    return sum((0.5 * (n + 1) * s) ** 2 for n, s in zip(dims, sp))


def random_vertex(rng, dims):
    ax = int(rng.integers(3))
    u = [float(rng.integers(0, n)) for n in dims]
    u[ax] = float(rng.integers(-1, dims[ax])) + 0.5
    return u


def threshold(F, R2):
    """T(F) from the doubled coefficients: the smallest value the exact
    maximum's pairs can take when some pair reached F."""
    alpha = 2.0 * 5.1 * U + 1e-14
    beta = 2.0 * 4.1 * U * np.sqrt(R2)
    gamma = 2.0 * max(20.2 * U * R2, 4.1 * U * U * R2)
    f = float(F)
    if not f > gamma:
        return 0.0
    a1 = 1.0 + alpha
    s = (-beta + np.sqrt(beta * beta + 4.0 * a1 * (f - gamma))) / (2.0 * a1)
    t = (1.0 - alpha) * s * s - beta * s - gamma
    if not t > 0:
        return 0.0
    x = np.float32(t)  # rounded toward minus infinity, as the kernels do
    if float(x) > t:
        x = np.nextafter(x, np.float32(-np.inf))
    return float(x)


@pytest.mark.parametrize("dims,sp", GRIDS)
def test_pair_error_bounds(dims, sp):
    rng = np.random.default_rng(5)
    R2 = radius2(dims, sp)
    R = np.sqrt(R2)
    pairs = []
    for _ in range(600):  # anywhere in the grid
        pairs.append((random_vertex(rng, dims), random_vertex(rng, dims)))
    for _ in range(300):  # short pairs far from the centre: the R^2 terms dominate
        a = random_vertex(rng, dims)
        for k in range(3):
            a[k] = (dims[k] - 1 - (a[k] % 3)) if rng.random() < 0.5 else (a[k] % 3)
        b = list(a)
        ax = int(rng.integers(3))
        b[ax] = a[ax] + float(rng.choice([-1.5, -1.0, -0.5, 0.5, 1.0, 1.5]))
        pairs.append((a, b))
    for _ in range(300):  # near-diametral pairs
        a = [float(rng.integers(0, 2)) for _ in range(3)]
        b = [dims[k] - 1 - float(rng.integers(0, 2)) for k in range(3)]
        ax = int(rng.integers(3))
        a[ax] -= 0.5
        b[ax] += 0.5 if rng.random() < 0.5 else -0.5
        pairs.append((a, b))
    worst_g = worst_f = 0.0
    for ua, ub in pairs:
        ea, eb = entry(ua, dims, sp), entry(ub, dims, sp)
        d2 = exact_d2(ua, ub, sp)
        sq = float(d2) ** 0.5
        g = Fraction(float(g_expansion(ea, eb)))
        f = Fraction(float(f_difference(ea, eb)))
        bound_g = 4.1 * U * R * sq + 20.2 * U * R2
        bound_f = 5.1 * U * float(d2) + 4.1 * U * R * sq + 4.1 * U * U * R2
        eg, ef = abs(float(g - d2)), abs(float(f - d2))
        assert eg <= bound_g, (ua, ub, eg, bound_g)
        assert ef <= bound_f, (ua, ub, ef, bound_f)
        worst_g, worst_f = max(worst_g, eg / bound_g), max(worst_f, ef / bound_f)
    # the bounds are not vacuous: with spacings that are not dyadic (0.7, 0.8 mm)
    # the observed errors reach a visible part of them; with dyadic spacings
    # every position and norm is exact in FP32 and so is the result
    if any(v not in (0.5, 1.0, 2.0) for v in sp):
        assert worst_g > 0.02 and worst_f > 0.02, (worst_g, worst_f)
    else:
        assert worst_g == 0.0 and worst_f == 0.0, (worst_g, worst_f)


@pytest.mark.parametrize("dims,sp", [GRIDS[0], GRIDS[2]])
def test_pair_error_bounds_soft_positions(dims, sp):
    """Soft maps: a vertex sits at owner + t along its edge with any FP64 t in
    (0, 1), so positions are not on the half-integer lattice; the same bounds
    hold (they only use |P| <= R)."""
    rng = np.random.default_rng(9)
    R2 = radius2(dims, sp)
    R = np.sqrt(R2)
    worst = 0.0
    for _ in range(800):
        uu = []
        for _v in range(2):
            ax = int(rng.integers(3))
            u = [float(rng.integers(0, n)) for n in dims]
            u[ax] = float(rng.integers(-1, dims[ax])) + float(rng.uniform(0.001, 0.999))
            uu.append(u)
        if rng.random() < 0.4:  # short pairs
            uu[1] = [uu[0][k] + float(rng.uniform(-1.5, 1.5)) for k in range(3)]
        ea, eb = entry(uu[0], dims, sp), entry(uu[1], dims, sp)
        d2 = exact_d2(uu[0], uu[1], sp)
        sq = float(d2) ** 0.5
        eg = abs(float(Fraction(float(g_expansion(ea, eb))) - d2))
        ef = abs(float(Fraction(float(f_difference(ea, eb))) - d2))
        bg = 4.1 * U * R * sq + 20.2 * U * R2
        bf = 5.1 * U * float(d2) + 4.1 * U * R * sq + 4.1 * U * U * R2
        assert eg <= bg and ef <= bf, (uu, eg, bg, ef, bf)
        worst = max(worst, eg / bg, ef / bf)
    assert worst > 0.02


@pytest.mark.parametrize("dims,sp", GRIDS[:2])
def test_threshold_keeps_every_maximal_pair(dims, sp):
    """Small vertex sets with many exact ties at the maximum (points on the
    corners of boxes): for F = the largest g or f of any pair, every pair
    attaining the exact maximum has both g and f >= T(F)."""
    rng = np.random.default_rng(11)
    R2 = radius2(dims, sp)
    for trial in range(6):
        lo = [float(rng.integers(0, n // 2 - 2)) for n in dims]
        hi = [float(rng.integers(n // 2 + 2, n)) for n in dims]
        verts = []
        for c in range(8):  # box corners, each as a vertex half a voxel off along x, y or z
            base = [hi[k] if (c >> k) & 1 else lo[k] for k in range(3)]
            for ax in range(3):
                v = list(base)
                v[ax] += 0.5 if (c >> ax) & 1 else -0.5
                verts.append(v)
        for _ in range(12):  # vertices strictly inside the box: shorter pairs
            v = [float(rng.integers(lo[k] + 1, hi[k])) for k in range(3)]
            v[int(rng.integers(3))] += 0.5
            verts.append(v)
        ent = [entry(v, dims, sp) for v in verts]
        d2 = {}
        gs, fs = {}, {}
        for i in range(len(verts)):
            for j in range(i + 1, len(verts)):
                d2[(i, j)] = exact_d2(verts[i], verts[j], sp)
                gs[(i, j)] = float(g_expansion(ent[i], ent[j]))
                fs[(i, j)] = float(f_difference(ent[i], ent[j]))
        dmax = max(d2.values())
        top = [p for p, v in d2.items() if v == dmax]
        assert len(top) >= 2  # ties at the maximum
        F = max(max(gs.values()), max(fs.values()))
        T = threshold(F, R2)
        assert T > 0.0
        for p in top:
            assert gs[p] >= T and fs[p] >= T, (trial, p, gs[p], fs[p], T)


def box_ub(alo, ahi, blo, bhi):
    """The culling bound of two boxes of FP32 positions, in the kernels' order:
    per axis the larger of fl(bhi - alo) and fl(ahi - blo), then
    fma(mz, mz, fma(my, my, fl(mx mx)))."""
    m = [max(np.float32(bhi[k] - alo[k]), np.float32(ahi[k] - blo[k])) for k in range(3)]
    f = np.float32(m[0] * m[0])
    f = fma32(m[1], m[1], f)
    return fma32(m[2], m[2], f)


@pytest.mark.parametrize("dims,sp", [GRIDS[0], GRIDS[2]])
def test_box_bound_covers_every_pair_without_epsilon(dims, sp):
    """Tiles of FP32 positions (near each other, overlapping, far apart): the
    culling bound of the two tiles' boxes is >= the difference-form f of every
    pair drawn from them, exactly (monotone FP32 operations)."""
    rng = np.random.default_rng(3)
    for trial in range(60):
        centre = [random_vertex(rng, dims) for _ in range(2)]
        if trial % 3 == 0:
            centre[1] = [c + float(rng.uniform(-3, 3)) for c in centre[0]]
        tiles = []
        for t in range(2):
            pts = []
            for _ in range(8):
                u = [centre[t][k] + float(rng.uniform(-4, 4)) for k in range(3)]
                pts.append(entry(u, dims, sp))
            lo = [min(p[0][k] for p in pts) for k in range(3)]
            hi = [max(p[0][k] for p in pts) for k in range(3)]
            tiles.append((pts, lo, hi))
        (pa, alo, ahi), (pb, blo, bhi) = tiles
        ub = box_ub(alo, ahi, blo, bhi)
        for ea in pa:
            for eb in pb:
                assert f_difference(ea, eb) <= ub and f_difference(eb, ea) <= ub
