"""Pins of the oracle's projection (Eq. 8), multiwavelet filters and MRA
(Eq. 9-10, Sect. 2.2 and 2.2.1) against facts fixed by the mathematics:
quadrature, orthogonality, closed-form filter entries, Parseval, lossless
round trips, brute-force active sets and the grid invariants."""
import numpy as np
import pytest

import oracle as O
from paper_2107_02750_gb300 import synth as S
from util import oracle_sim

S3 = np.sqrt(3.0)
GX, GW = np.polynomial.legendre.leggauss(4)   # exact for the polynomials used here
GX = 0.5 * GX                                   # nodes on [-1/2, 1/2]
GW = 0.5 * GW


def bilinear_projection(vert):
    """L2 projection of the bilinear vertex interpolant on [1, 2 sqrt3 x, 2 sqrt3 y]
    by tensor Gauss quadrature (average-normalised coefficients)."""
    ny, nx = vert.shape[0] - 1, vert.shape[1] - 1
    c = np.zeros((3, ny, nx))
    for a, wa in zip(GX, GW):
        for b, wb in zip(GX, GW):
            s, t = a + 0.5, b + 0.5
            f = ((1 - s) * (1 - t) * vert[:-1, :-1] + s * (1 - t) * vert[:-1, 1:]
                 + (1 - s) * t * vert[1:, :-1] + s * t * vert[1:, 1:])
            w = wa * wb
            c[0] += w * f
            c[1] += w * f * 2 * S3 * a
            c[2] += w * f * 2 * S3 * b
    return c


def test_projection_is_l2_projection_of_bilinear_interpolant():
    rng = np.random.default_rng(11)
    vert = rng.normal(size=(9, 13))
    got = np.array(O.project(vert))
    want = bilinear_projection(vert)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


def test_projection_of_a_plane_is_exact():
    y, x = np.mgrid[0:6, 0:8].astype(float)
    vert = 3.0 + 0.7 * x - 1.3 * y
    c0, c1x, c1y = O.project(vert)
    np.testing.assert_allclose(c0, 3.0 + 0.7 * (np.arange(7) + 0.5)[None, :] - 1.3 * (np.arange(5) + 0.5)[:, None], atol=1e-14)
    np.testing.assert_allclose(c1x, 0.7 / (2 * S3), atol=1e-15)
    np.testing.assert_allclose(c1y, -1.3 / (2 * S3), atol=1e-15)


def _Q():
    A, G = O.filters()
    Q = np.zeros((12, 12))
    for c in range(4):
        Q[0:3, 3 * c:3 * c + 3] = 0.5 * A[c]
        Q[3:12, 3 * c:3 * c + 3] = G[c]
    return A, G, Q


def test_filter_bank_is_orthogonal():
    _, _, Q = _Q()
    np.testing.assert_allclose(Q @ Q.T, np.eye(12), atol=1e-14)


def test_highpass_closed_form():
    """The projected Haar x basis vectors are already mutually orthogonal, so
    the symmetric orthonormalisation is a normalisation; entries in closed
    form (rows: H,V,D x (1, x-slope, y-slope); child c = ix + 2 iy)."""
    _, G, _ = _Q()
    for c in range(4):
        sx = 1 if c & 1 else -1
        sy = 1 if c & 2 else -1
        want = np.zeros((9, 3))
        want[0] = [0.25 * sy, 0.0, -S3 / 4]     # H, average
        want[1] = [0.0, 0.5 * sy, 0.0]          # H, x-slope
        want[2] = [0.0, 0.0, 0.5 * sy]          # H, y-slope
        want[3] = [0.25 * sx, -S3 / 4, 0.0]     # V, average
        want[4] = [0.0, 0.5 * sx, 0.0]
        want[5] = [0.0, 0.0, 0.5 * sx]
        want[6] = [0.5 * sx * sy, 0.0, 0.0]     # D, average
        want[7] = [0.0, 0.5 * sx * sy, 0.0]
        want[8] = [0.0, 0.0, 0.5 * sx * sy]
        np.testing.assert_allclose(G[c], want, atol=1e-14)


def _piecewise_planar(children, a, b):
    """value of the child planes at parent-local point (a, b) in [-1/2,1/2]^2"""
    ix = (a > 0).astype(int)
    iy = (b > 0).astype(int)
    c = ix + 2 * iy
    xc = 2 * (a - np.where(ix, 0.25, -0.25))
    yc = 2 * (b - np.where(iy, 0.25, -0.25))
    s = children[c]
    return s[..., 0] + 2 * S3 * xc * s[..., 1] + 2 * S3 * yc * s[..., 2]


def test_parent_row_is_quadrature_projection():
    rng = np.random.default_rng(5)
    ch = rng.normal(size=(4, 3))
    sp, _ = O.encode_node(ch)
    want = np.zeros(3)
    for q in range(4):   # each child quadrant separately (piecewise smooth)
        ox = 0.25 if q & 1 else -0.25
        oy = 0.25 if q & 2 else -0.25
        for a, wa in zip(GX, GW):
            for b, wb in zip(GX, GW):
                A = ox + 0.5 * a
                B = oy + 0.5 * b
                f = _piecewise_planar(ch, np.array(A), np.array(B))
                w = 0.25 * wa * wb
                want += w * np.array([f, f * 2 * S3 * A, f * 2 * S3 * B])
    np.testing.assert_allclose(sp, want, atol=1e-13)


def test_parseval_and_lossless_round_trip():
    rng = np.random.default_rng(7)
    for _ in range(20):
        ch = rng.normal(size=(4, 3))
        sp, d = O.encode_node(ch)
        assert abs(0.25 * np.sum(ch ** 2) - (np.sum(sp ** 2) + 0.25 * np.sum(d ** 2))) < 1e-13
        np.testing.assert_allclose(O.decode_node(sp, d), ch, atol=1e-14)


def test_plane_has_zero_details():
    rng = np.random.default_rng(9)
    p = rng.normal(size=3)
    ch = np.array([[p[0] + S3 / 2 * (1 if c & 1 else -1) * p[1] + S3 / 2 * (1 if c & 2 else -1) * p[2],
                    0.5 * p[1], 0.5 * p[2]] for c in range(4)])
    sp, d = O.encode_node(ch)
    np.testing.assert_allclose(sp, p, atol=1e-15)
    assert np.abs(d).max() < 1e-15


def test_lossless_multilevel_decode_circular_dam_break_128():
    """Dam-break initial state at L = 7, epsilon = 0: encode to level 0 and
    decode back (one MWDG2 adaptation) reproduces the finest coefficients."""
    p = S.dam_break_circular(L=7, eps=0.0, mode=S.ADAPTIVE)
    s = oracle_sim(p)
    lev0, i0, j0, c0 = s.leaves()
    s.adapt()
    lev, i, j, c = s.leaves()
    assert (lev == 7).all() and len(lev) == 128 * 128
    np.testing.assert_array_equal(i, i0)
    np.testing.assert_array_equal(j, j0)
    err = np.abs(c - c0).max() / np.abs(c0).max()
    assert err <= 1e-13


def _leaf_cover(lev, i, j, L, nx, ny):
    cover = np.zeros((ny, nx), int)
    for l, a, b in zip(lev, i, j):
        w = 1 << (L - l)
        cover[b * w:(b + 1) * w, a * w:(a + 1) * w] += 1
    return cover


def _finest_level_map(lev, i, j, L, nx, ny):
    m = np.zeros((ny, nx), int)
    for l, a, b in zip(lev, i, j):
        w = 1 << (L - l)
        m[b * w:(b + 1) * w, a * w:(a + 1) * w] = l
    return m


def quadrature_details(zc, zs, L):
    """normalised topography detail per node from a direct evaluation of the
    nine detail basis functions (closed form) against the finest planes by
    quadrature; independent of the filter code"""
    out = {}
    ny, nx = zc.shape
    norm = max(1.0, np.abs(zc).max())
    for l in range(L):
        w = 1 << (L - l)
        nyl, nxl = ny // w, nx // w
        dm = np.zeros((nyl, nxl))
        for jj in range(nyl):
            for ii in range(nxl):
                blk0 = zc[jj * w:(jj + 1) * w, ii * w:(ii + 1) * w]
                blkx = zs[0][jj * w:(jj + 1) * w, ii * w:(ii + 1) * w]
                blky = zs[1][jj * w:(jj + 1) * w, ii * w:(ii + 1) * w]
                # the node's 4 children as planes: encode their finest content
                # by exact averaging (average and first moments of planes)
                half = w // 2
                ch = np.zeros((4, 3))
                for c in range(4):
                    sl = (slice((c >> 1) * half, (c >> 1) * half + half),
                          slice((c & 1) * half, (c & 1) * half + half))
                    # finest cell centres relative to the child, in child units
                    yy, xx = np.mgrid[0:half, 0:half]
                    xr = (xx + 0.5) / half - 0.5
                    yr = (yy + 0.5) / half - 0.5
                    b0, bx, by = blk0[sl], blkx[sl], blky[sl]
                    ch[c, 0] = b0.mean()
                    # first moments: <f, 2 sqrt3 x_child> over the child
                    ch[c, 1] = np.mean(b0 * 2 * S3 * xr + bx / half)
                    ch[c, 2] = np.mean(b0 * 2 * S3 * yr + by / half)
                dets = []
                for c in range(4):
                    sx = 1 if c & 1 else -1
                    sy = 1 if c & 2 else -1
                    dets.append([0.25 * sy * ch[c, 0] - S3 / 4 * ch[c, 2], 0.5 * sy * ch[c, 1], 0.5 * sy * ch[c, 2],
                                 0.25 * sx * ch[c, 0] - S3 / 4 * ch[c, 1], 0.5 * sx * ch[c, 1], 0.5 * sx * ch[c, 2],
                                 0.5 * sx * sy * ch[c, 0], 0.5 * sx * sy * ch[c, 1], 0.5 * sx * sy * ch[c, 2]])
                d = np.sum(np.array(dets), axis=0)
                dm[jj, ii] = np.abs(d).max() / norm
        out[l] = dm
    return out


@pytest.mark.parametrize("eps", [1e-3, 1e-2, 5e-2])
def test_active_set_brute_force_tiny_grid(eps):
    """Static grid without grading: the nodes flagged by brute force (quadrature
    details >= eps, closed under parents) give exactly the oracle's leaves;
    grading only adds refinement."""
    L = 4
    rng = np.random.default_rng(3)
    nx = ny = 16
    y, x = np.mgrid[0:ny + 1, 0:nx + 1].astype(float)
    vert = 0.3 * x + np.exp(-((x - 5) ** 2 + (y - 11) ** 2) / 6.0) * 2 + 0.02 * rng.normal(size=x.shape)
    zc, zx, zy = bilinear_projection(vert)
    dets = quadrature_details(zc, (zx, zy), L)
    flag = {l: dets[l] >= eps for l in range(L)}
    for l in range(L - 1, 0, -1):
        f = flag[l]
        up = f.reshape(f.shape[0] // 2, 2, f.shape[1] // 2, 2).any(axis=(1, 3))
        flag[l - 1] = flag[l - 1] | up
    want = []
    for l in range(L + 1):
        nl = 1 << l
        for jj in range(nl):
            for ii in range(nl):
                f = flag[l][jj, ii] if l < L else False
                parent = True if l == 0 else flag[l - 1][jj // 2, ii // 2]
                if parent and not f:
                    want.append((l, ii, jj))
    # oracle's static grid without grading is read through its z details
    p = S.Problem("tiny", 1, 1, L, 1.0, vert, np.zeros_like(vert), np.zeros_like(vert),
                  np.zeros_like(vert), eps=eps, mode=S.STATIC)
    s = oracle_sim(p)
    for l in range(L):
        _, dz = s.z_level(l)
        np.testing.assert_allclose(dz.reshape(1 << l, 1 << l), dets[l], atol=1e-12)
    lev, ii, jj, _ = s.leaves()
    got = set(zip(lev.tolist(), ii.tolist(), jj.tolist()))
    # grading refines further: every brute-force leaf is covered by leaves at
    # the same level or finer
    fmap = _finest_level_map(lev, ii, jj, L, nx, ny)
    for (l, a, b) in want:
        w = 1 << (L - l)
        assert (fmap[b * w:(b + 1) * w, a * w:(a + 1) * w] >= l).all()
    assert len(got) >= len(want)


def _check_tiling_and_grading(s, p, graded=True):
    lev, i, j, _ = s.leaves()
    L = p.L
    cover = _leaf_cover(lev, i, j, L, p.nx, p.ny)
    assert (cover == 1).all(), "leaves must partition the domain"
    if graded:
        m = _finest_level_map(lev, i, j, L, p.nx, p.ny)
        assert np.abs(np.diff(m, axis=0)).max() <= 1
        assert np.abs(np.diff(m, axis=1)).max() <= 1
    return lev


def test_static_grid_invariants_on_valley_terrain():
    p = S.valley(n=128, L=7, mode=S.STATIC, eps=1e-3)
    s = oracle_sim(p)
    lev = _check_tiling_and_grading(s, p)
    assert 0 < len(lev) < 128 * 128


def test_epsilon_limits():
    p = S.valley(n=64, L=6, mode=S.STATIC, eps=0.0)
    s = oracle_sim(p)
    lev = _check_tiling_and_grading(s, p)
    assert (lev == 6).all() and len(lev) == 64 * 64
    p = S.valley(n=64, L=6, mode=S.STATIC, eps=1e9)
    s = oracle_sim(p)
    lev = _check_tiling_and_grading(s, p)
    assert (lev == 0).all() and len(lev) == 1


def test_planar_dem_collapses_to_coarsest():
    y, x = np.mgrid[0:65, 0:65].astype(float)
    vert = 5.0 + 0.1 * x - 0.05 * y
    p = S.Problem("plane", 2, 2, 5, 1.0, vert, np.zeros_like(vert), np.zeros_like(vert),
                  np.zeros_like(vert), eps=1e-6, mode=S.STATIC)
    s = oracle_sim(p)
    lev = _check_tiling_and_grading(s, p)
    assert (lev == 0).all() and len(lev) == 4


def test_grading_is_minimal_on_tiny_grid():
    """Every refined node of the graded static grid is justified: its own
    quadrature detail reaches epsilon, one of its children is refined
    (closure), or it is the parent of a face neighbour of a refined node one
    level finer (2:1 grading)."""
    L, eps = 4, 1e-3
    y, x = np.mgrid[0:17, 0:17].astype(float)
    vert = 3 * np.exp(-((x - 3) ** 2 + (y - 3) ** 2) / 2.0)
    p = S.Problem("g", 1, 1, L, 1.0, vert, np.zeros_like(vert), np.zeros_like(vert),
                  np.zeros_like(vert), eps=eps, mode=S.STATIC)
    s = oracle_sim(p)
    lev, i, j, _ = s.leaves()
    m = _finest_level_map(lev, i, j, L, 16, 16)
    assert np.abs(np.diff(m, axis=0)).max() <= 1 and np.abs(np.diff(m, axis=1)).max() <= 1
    sig = {}
    for l in range(L):
        w = 1 << (L - l)
        sig[l] = m.reshape(16 // w, w, 16 // w, w).max(axis=(1, 3)) > l
    zc, zx, zy = bilinear_projection(vert)
    dets = quadrature_details(zc, (zx, zy), L)
    added = 0
    for l in range(L):
        nl = 1 << l
        for jj in range(nl):
            for ii in range(nl):
                if not sig[l][jj, ii]:
                    continue
                ok = dets[l][jj, ii] >= eps
                if l + 1 < L:
                    ok = ok or sig[l + 1][2 * jj:2 * jj + 2, 2 * ii:2 * ii + 2].any()
                    n2 = 1 << (l + 1)
                    for b in range(n2):
                        for a in range(n2):
                            if not sig[l + 1][b, a]:
                                continue
                            for da, db in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                                na, nb = a + da, b + db
                                if 0 <= na < n2 and 0 <= nb < n2 and (na // 2, nb // 2) == (ii, jj):
                                    ok = True
                if dets[l][jj, ii] < eps:
                    added += 1
                assert ok, (l, ii, jj)
    assert added > 0


def test_projection_matches_the_printed_eq8_examples():
    """tests/golden/eq8_projection.txt: one element per line, its four
    vertex heights and the planes evaluated by hand from Eq. 8a-c."""
    import math
    from pathlib import Path
    import numpy as np
    import oracle as O
    rows = []
    for line in (Path(__file__).parent / "golden" / "eq8_projection.txt").read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        verts, z0, nums = (part.split() for part in line.split("|"))
        rows.append(([float(v) for v in verts], float(z0[0]), [float(x) for x in nums]))
    assert len(rows) >= 5
    for (sw, se, nw, ne), z0, (nx_, ny_) in rows:
        vert = np.array([[sw, se], [nw, ne]])      # row j = 0 south, j = 1 north
        c0, c1x, c1y = O.project(vert)
        assert abs(c0[0, 0] - z0) <= 1e-15 * max(1.0, abs(z0))
        assert abs(c1x[0, 0] - nx_ / (4.0 * math.sqrt(3.0))) <= 1e-15
        assert abs(c1y[0, 0] - ny_ / (4.0 * math.sqrt(3.0))) <= 1e-15


@pytest.mark.parametrize("eps", [1e-2, 3e-2, 1e-1])
def test_mwdg2_adaptation_brute_force_tiny_grid(eps):
    """MWDG2 regridding (Sect. 2.3, Eq. 9 and the normalised details of
    Sect. 2.2) from all-finest leaves, by brute force: each node's measure
    is the largest of its topography detail and its flow details (h, qx,
    qy), each divided by max(1, max |v0|) over the current leaves, with the
    details from a direct quadrature of the finest planes (independent of
    the filter code); a node is significant when the measure reaches eps,
    its eight same-level neighbours are flagged too (prediction), parents of
    flagged nodes are flagged (closure), and the leaves are the unflagged
    children of flagged nodes (or the root).  The oracle's leaves after one
    adaptation must be exactly these."""
    L, n = 4, 16
    rng = np.random.default_rng(17)
    y, x = np.mgrid[0:n + 1, 0:n + 1].astype(float)
    z = 0.05 * x + 0.8 * np.exp(-((x - 4) ** 2 + (y - 12) ** 2) / 5.0) + 1e-5 * rng.normal(size=x.shape)
    h = 1.0 + 0.6 * np.exp(-((x - 11) ** 2 + (y - 5) ** 2) / 3.0) + 1e-5 * rng.normal(size=x.shape)
    qx = 0.3 * np.tanh((x - 8) / 1.5) + 1e-5 * rng.normal(size=x.shape)
    qy = 0.2 * np.exp(-((x - 12) ** 2 + (y - 12) ** 2) / 4.0)
    measure = {l: np.zeros((1 << l, 1 << l)) for l in range(L)}
    for v in (z, h, qx, qy):
        c = bilinear_projection(v)
        d = quadrature_details(c[0], (c[1], c[2]), L)
        for l in range(L):
            measure[l] = np.maximum(measure[l], d[l])
    gap = min(np.abs(measure[l] - eps).min() for l in range(L))
    assert gap > 1e-9, gap  # no decision within rounding of eps
    flag = {}
    for l in range(L):
        f0 = measure[l] >= eps
        f = f0.copy()
        nl = 1 << l
        for jj, ii in zip(*np.nonzero(f0)):
            f[max(jj - 1, 0):min(jj + 2, nl), max(ii - 1, 0):min(ii + 2, nl)] = True
        flag[l] = f
    for l in range(L - 1, 0, -1):
        f = flag[l]
        flag[l - 1] = flag[l - 1] | f.reshape(f.shape[0] // 2, 2, f.shape[1] // 2, 2).any(axis=(1, 3))
    want = set()
    for l in range(L + 1):
        for jj in range(1 << l):
            for ii in range(1 << l):
                f = flag[l][jj, ii] if l < L else False
                parent = True if l == 0 else flag[l - 1][jj // 2, ii // 2]
                if parent and not f:
                    want.add((l, ii, jj))
    s = O.Sim(M=1, N=1, L=L, R=1.0, mode=S.ADAPTIVE, eps=eps)
    s.load_dem(z)
    s.load_roughness(np.zeros((n, n)))
    s.load_initial(h, qx, qy)
    s.init_grid()
    s.adapt()
    lev, ii, jj, _ = s.leaves()
    got = set(zip(lev.tolist(), ii.tolist(), jj.tolist()))
    assert got == want, (sorted(got - want)[:5], sorted(want - got)[:5])
    assert 2 <= len(np.unique(lev)) and len(got) < n * n
