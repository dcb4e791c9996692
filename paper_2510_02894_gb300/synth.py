"""Seeded synthetic inputs shaped like the CT/MRI regions of interest the paper
measures on (KITS19 kidney/tumour masks, Sec. 3; the dataset itself is not
available, so these stand in for it).

This module holds input generation only -- none of the shape-feature
arithmetic.  Both the CUDA path and the CPU oracle consume its arrays.
Arrays are C-order [nz][ny][nx] (x fastest); spacing is (sx, sy, sz) in mm.

Workloads (all seeded with numpy.random.default_rng):
  ellipsoid_32   32^3 uint8, axis-aligned solid ellipsoid, semi-axes (10, 7, 5)
  ct_512         512x512x256 uint8, union of 3 rotated ellipsoids, 5 % of the
                 boundary voxels flipped, spacing (0.7, 0.7, 2.5)
  batch_256      256 crops with log-normal edges in [16, 192], ellipsoids or
                 thresholded smoothed-noise blobs, three spacings
  soft_160       160^3 float32 probability map, sigmoid of smoothed signed
                 distance logits of a rotated ellipsoid
  blobs_512x8    8 x 512^3 uint8 smoothed-noise blobs filling ~40 %, spacing
                 (0.6, 0.6, 1.2)
"""
import numpy as np

SPACINGS_BATCH = ((1.0, 1.0, 1.0), (0.8, 0.8, 3.0), (0.5, 0.5, 1.0))


def random_rotation(rng):
    """Uniform rotation from the QR factorisation of a Gaussian matrix."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def ellipsoid(shape_zyx, centre_xyz, semi_xyz, rot=None, out=None):
    """Boolean solid ellipsoid: inside iff |diag(1/a) R^T (x - c)|^2 <= 1,
    evaluated at voxel centres (integer index coordinates)."""
    nz, ny, nx = shape_zyx
    if out is None:
        out = np.zeros(shape_zyx, dtype=bool)
    rot = np.eye(3) if rot is None else np.asarray(rot, np.float64)
    c = np.asarray(centre_xyz, np.float64)
    inv_a = 1.0 / np.asarray(semi_xyz, np.float64)
    m = (rot * inv_a[None, :])  # columns scaled: local_k = sum_j R[j,k] d_j / a_k
    xs = np.arange(nx, dtype=np.float64) - c[0]
    ys = np.arange(ny, dtype=np.float64) - c[1]
    for z in range(nz):
        dz = z - c[2]
        # local coordinates, shape (ny, nx) per component
        acc = np.zeros((ny, nx))
        for k in range(3):
            lk = (xs[None, :] * m[0, k] + ys[:, None] * m[1, k]) + dz * m[2, k]
            acc += lk * lk
        out[z] |= acc <= 1.0
    return out


def _gaussian(field, sigma):
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(field, sigma=sigma, mode="constant", truncate=4.0)


def ellipsoid_32(seed=0):
    """Config: one 32^3 mask, axis-aligned ellipsoid (10, 7, 5), centre offset
    uniform in [-3, 3] per axis, spacing (1, 1, 1)."""
    rng = np.random.default_rng(seed)
    centre = 15.5 + rng.uniform(-3.0, 3.0, size=3)
    mask = ellipsoid((32, 32, 32), centre, (10.0, 7.0, 5.0)).astype(np.uint8)
    return mask, (1.0, 1.0, 1.0)


def boundary_voxels(mask):
    """Voxels with a 6-neighbour of the other label (outside the grid is 0)."""
    m = mask.astype(bool)
    p = np.pad(m, 1)
    b = np.zeros_like(m)
    for ax in range(3):
        for sh in (-1, 1):
            nb = np.roll(p, sh, axis=ax)[1:-1, 1:-1, 1:-1]
            b |= nb != m
    return b


def ct_512(seed=0, shape_zyx=(256, 512, 512), flip_frac=0.05):
    """Config: 512x512x256 uint8 CT-shaped mask, spacing (0.7, 0.7, 2.5): union
    of 3 ellipsoids (semi-axes uniform 60-150 voxels, uniform random rotation,
    centres uniform in the volume), then 5 % of the boundary voxels flipped."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape_zyx
    mask = np.zeros(shape_zyx, dtype=bool)
    scale = min(nx, ny, nz) / 256.0
    for _ in range(3):
        semi = rng.uniform(60.0, 150.0, size=3) * scale
        rot = random_rotation(rng)
        centre = rng.uniform(0.0, 1.0, size=3) * np.array([nx - 1, ny - 1, nz - 1])
        ellipsoid(shape_zyx, centre, semi, rot, out=mask)
    b = boundary_voxels(mask)
    idx = np.flatnonzero(b)
    flip = idx[rng.random(idx.size) < flip_frac]
    flat = mask.reshape(-1)
    flat[flip] = ~flat[flip]
    return mask.astype(np.uint8), (0.7, 0.7, 2.5)


def _noise_blob(rng, shape_zyx, sigma, window=True):
    noise = rng.random(shape_zyx)
    sm = _gaussian(noise, sigma)
    if window:
        nz, ny, nx = shape_zyx
        zz = (np.arange(nz) - (nz - 1) / 2.0) / (nz / 2.0)
        yy = (np.arange(ny) - (ny - 1) / 2.0) / (ny / 2.0)
        xx = (np.arange(nx) - (nx - 1) / 2.0) / (nx / 2.0)
        r2 = zz[:, None, None] ** 2 + yy[None, :, None] ** 2 + xx[None, None, :] ** 2
        sm = sm * np.clip(1.0 - r2, 0.0, 1.0)
    lo, hi = sm.min(), sm.max()
    return (sm - lo) / (hi - lo if hi > lo else 1.0)


def batch_256(seed=0, n=256):
    """Config: n crops; edge per axis log-normal (median 55.4, sigma 0.62)
    clipped to [16, 192]; each a rotated ellipsoid (semi-axes 0.25-0.45 of the
    edge) or a Gaussian-smoothed noise blob (sigma 2-6) in a radial window,
    min-max normalised and thresholded at 0.5; spacing drawn from three CT/MRI
    spacings.  Returns a list of (mask, spacing)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        edges = np.clip(np.rint(rng.lognormal(np.log(55.4), 0.62, size=3)), 16, 192).astype(int)
        nx, ny, nz = (int(e) for e in edges)
        sp = SPACINGS_BATCH[int(rng.integers(0, len(SPACINGS_BATCH)))]
        if rng.random() < 0.5:
            semi = rng.uniform(0.25, 0.45, size=3) * edges
            centre = (edges - 1) / 2.0
            m = ellipsoid((nz, ny, nx), centre, semi, random_rotation(rng)).astype(np.uint8)
        else:
            sigma = rng.uniform(2.0, 6.0)
            m = (_noise_blob(rng, (nz, ny, nx), sigma) > 0.5).astype(np.uint8)
        out.append((np.ascontiguousarray(m), sp))
    return out


def soft_160(seed=0, n=160):
    """Config: n^3 float32 probability map = sigmoid(4 * G_3(sd)), sd the
    approximate signed distance (positive inside) of a rotated ellipsoid with
    semi-axes uniform 30-60 voxels and centre 79.5 + U[-5, 5]:
    sd(x) = (1 - |diag(1/a) R^T (x - c)|) * min(a)."""
    rng = np.random.default_rng(seed)
    scale = n / 160.0
    semi = rng.uniform(30.0, 60.0, size=3) * scale
    rot = random_rotation(rng)
    centre = (n - 1) / 2.0 + rng.uniform(-5.0, 5.0, size=3) * scale
    g = np.arange(n, dtype=np.float64)
    d = [g - centre[k] for k in range(3)]
    X = d[0][None, None, :]
    Y = d[1][None, :, None]
    Z = d[2][:, None, None]
    acc = np.zeros((n, n, n))
    for k in range(3):
        lk = (X * rot[0, k] + Y * rot[1, k] + Z * rot[2, k]) / semi[k]
        acc = acc + lk * lk
    sd = (1.0 - np.sqrt(acc)) * semi.min()
    logits = 4.0 * _gaussian(sd, 3.0 * scale)
    prob = 1.0 / (1.0 + np.exp(-logits))
    return prob.astype(np.float32), (1.0, 1.0, 1.0)


def blobs_512(seed=0, count=8, n=512, fill=0.40):
    """Config: `count` masks of n^3 uint8, each a smoothed-noise blob in a
    radial window thresholded at its (1 - fill) quantile, spacing
    (0.6, 0.6, 1.2).  The noise is drawn on an n/8 grid, smoothed there and
    upsampled trilinearly, which keeps generation to seconds per mask."""
    from scipy.ndimage import zoom
    rng = np.random.default_rng(seed)
    out = []
    f = 8
    c = n // f
    for _ in range(count):
        coarse = _noise_blob(rng, (c, c, c), 1.2, window=True)
        full = zoom(coarse.astype(np.float32), f, order=1)
        thr = np.quantile(full[::4, ::4, ::4], 1.0 - fill)
        out.append((np.ascontiguousarray((full > thr).astype(np.uint8)), (0.6, 0.6, 1.2)))
    return out
