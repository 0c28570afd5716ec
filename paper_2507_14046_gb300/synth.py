"""Seeded synthetic workloads for the D²IP fitting path.

The paper's own data (COMSOL thorax sequences and clinical recordings, Sec. IV-A/B) are not
available, so every workload is synthetic and generated here from a seed:

* ``sensitivity_raw``  -- the un-normalised sensitivity matrix J (M x V) of the linearised
  forward model V = J Sigma (Eq. 1).  Rows are i.i.d. N(0,1) voxel fields smoothed by a
  truncated 3D Gaussian and damped with distance from the electrode ring they belong to.
* ``ellipsoid_phantom`` / ``breathing_amplitude`` -- ground-truth conductivity changes.
* ``measurements``     -- Delta v = J_n Delta sigma + Gaussian noise at a given SNR
  (noise robustness study, Sec. V-A), where J_n is the column-normalised J.  This is the
  data simulator; the fitting method normalises J independently.
* ``input_noise``      -- the fixed network input Z of Eq. 2 (N(0, 0.1^2), 8 channels, NDHWC).
* ``kaiming_theta``    -- Kaiming-normal initial weights (UPWS starts from them, Sec. III-B).

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea, Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), turned into uniforms by
taking the top 53 bits and into normals by the Box-Muller transform, so every value is a
pure function of (seed, stream, index) on any machine and NumPy version.

Everything is float64 internally; the arrays handed to the GPU library are float32, and
tests feed the same float32 values (widened) to the oracle.

This module holds none of the fitting method's arithmetic and imports nothing else from
the package; the oracle and the CUDA path both consume its arrays.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream ids: one per kind of random draw
STREAM_J = 1
STREAM_NOISE = 2
STREAM_Z = 3
STREAM_THETA = 4
STREAM_PHANTOM = 5
STREAM_BATCH = 6

MEAS_PER_RING = 16 * 13  # 16 electrodes, adjacent drive: 16 drives x 13 measurements


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrap-around arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    k = _mix64(s)
    k = _mix64(k ^ np.array([stream & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))
    return k[0]


def random_u64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """The SplitMix64 sequence started from state key(seed, stream): value i is
    mix64(key + (offset + i + 1) * gamma)."""
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        st = np.uint64(_key(seed, stream)) + idx * _GAMMA
    return _mix64(st)


def uniform(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniforms in the open interval (0, 1): (top 53 bits + 0.5) * 2^-53."""
    u = random_u64(seed, stream, count, offset) >> np.uint64(11)
    return (u.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    npair = (count + 1) // 2
    u = uniform(seed, stream, 2 * npair, 2 * offset)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * npair, dtype=np.float64)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:count]


# --------------------------------------------------------------------------------------
# Sensitivity matrix
# --------------------------------------------------------------------------------------

def gaussian_taps(sigma: float = 1.5, radius: int = 4) -> np.ndarray:
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    w = np.exp(-0.5 * (t / sigma) ** 2)
    return w / w.sum()


def _smooth_axis(a: np.ndarray, taps: np.ndarray, axis: int) -> np.ndarray:
    """Zero-padded correlation of ``a`` with symmetric ``taps`` along ``axis``."""
    r = (len(taps) - 1) // 2
    pad = [(0, 0)] * a.ndim
    pad[axis] = (r, r)
    ap = np.pad(a, pad)
    out = np.zeros_like(a)
    n = a.shape[axis]
    for k, w in enumerate(taps):
        sl = [slice(None)] * a.ndim
        sl[axis] = slice(k, k + n)
        out += w * ap[tuple(sl)]
    return out


def ring_planes(Z: int, rings: int) -> np.ndarray:
    """Plane coordinate of each electrode ring: Z * (k+1) / (rings+1)."""
    return np.array([Z * (k + 1) / (rings + 1) for k in range(rings)], dtype=np.float64)


def ring_decay(Z: int, rings: int, length: float = 3.0) -> np.ndarray:
    """exp(-|z_c - z_ring| / length) per (ring, plane), z_c = z + 0.5."""
    zc = np.arange(Z, dtype=np.float64) + 0.5
    zr = ring_planes(Z, rings)
    return np.exp(-np.abs(zc[None, :] - zr[:, None]) / length)


def sensitivity_raw(grid: tuple[int, int, int], rings: int, seed: int,
                    sigma: float = 1.5, radius: int = 4, chunk: int = 32,
                    decay: bool = True) -> np.ndarray:
    """Un-normalised J, float32, shape (rings*208, X*Y*Z), row-major.

    Rows are ordered ring-major (then 16 drives x 13 measurements).  Row i is an i.i.d.
    N(0,1) field over the grid, smoothed by a separable Gaussian (zero padding), times the
    decay of its ring (``decay=False`` leaves it out).  Column index q = (z*Y + y)*X + x.
    """
    X, Y, Z = grid
    m = rings * MEAS_PER_RING
    n = X * Y * Z
    taps = gaussian_taps(sigma, radius)
    dec = ring_decay(Z, rings)
    out = np.empty((m, n), dtype=np.float32)
    for r0 in range(0, m, chunk):
        r1 = min(m, r0 + chunk)
        g = normal(seed, STREAM_J, (r1 - r0) * n, offset=r0 * n).reshape(r1 - r0, Z, Y, X)
        for ax in (1, 2, 3):
            g = _smooth_axis(g, taps, ax)
        if decay:
            ring = np.arange(r0, r1) // MEAS_PER_RING
            g *= dec[ring][:, :, None, None]
        out[r0:r1] = g.reshape(r1 - r0, n).astype(np.float32)
    return out


# --------------------------------------------------------------------------------------
# Phantoms and measurements
# --------------------------------------------------------------------------------------

@dataclass(frozen=True)
class Ellipsoid:
    centre: tuple[float, float, float]   # (x, y, z) in voxel units, voxel centres at i+0.5
    semi: tuple[float, float, float]     # semi-axes (x, y, z)


def lung_pair(grid: tuple[int, int, int]) -> list[Ellipsoid]:
    """Two 'lungs' at (0.3X, 0.5Y, 0.5Z) and (0.7X, 0.5Y, 0.5Z), semi-axes (4,3,3)*X/16."""
    X, Y, Z = grid
    s = X / 16.0
    semi = (4.0 * s, 3.0 * s, 3.0 * s)
    return [Ellipsoid((0.3 * X, 0.5 * Y, 0.5 * Z), semi),
            Ellipsoid((0.7 * X, 0.5 * Y, 0.5 * Z), semi)]


def random_ellipsoids(grid: tuple[int, int, int], seed: int, problem: int,
                      count: int = 2) -> list[Ellipsoid]:
    """``count`` ellipsoids with semi-axes U[2,8] (capped to fit) and centres drawn so the
    whole ellipsoid lies inside the grid."""
    X, Y, Z = grid
    dims = (X, Y, Z)
    u = uniform(seed, STREAM_PHANTOM, 6 * count, offset=64 * problem)
    out = []
    for e in range(count):
        semi, cen = [], []
        for a in range(3):
            s = min(2.0 + 6.0 * u[6 * e + a], dims[a] / 2.0)
            lo, hi = s, dims[a] - s
            cen.append(lo + (hi - lo) * u[6 * e + 3 + a])
            semi.append(s)
        out.append(Ellipsoid(tuple(cen), tuple(semi)))
    return out


def ellipsoid_phantom(grid: tuple[int, int, int], ellipsoids: list[Ellipsoid],
                      value: float = -0.3) -> np.ndarray:
    """Delta sigma (float64, length X*Y*Z, index (z*Y+y)*X+x): ``value`` inside any ellipsoid."""
    X, Y, Z = grid
    z, y, x = np.meshgrid(np.arange(Z) + 0.5, np.arange(Y) + 0.5, np.arange(X) + 0.5,
                          indexing="ij")
    inside = np.zeros((Z, Y, X), dtype=bool)
    for e in ellipsoids:
        (cx, cy, cz), (ax, ay, az) = e.centre, e.semi
        inside |= ((x - cx) / ax) ** 2 + ((y - cy) / ay) ** 2 + ((z - cz) / az) ** 2 <= 1.0
    return np.where(inside, value, 0.0).reshape(-1)


def breathing_amplitude(T: int, period: float = 20.0) -> np.ndarray:
    """(1 + sin(2 pi t / period)) / 2 for t = 0..T-1 (0 at t = 15 for period 20)."""
    t = np.arange(T, dtype=np.float64)
    return (1.0 + np.sin(2.0 * math.pi * t / period)) / 2.0


def column_normalised(J32: np.ndarray) -> np.ndarray:
    """The simulator's own column-normalised copy of J (float64), used to synthesise data."""
    J = J32.astype(np.float64)
    return J / np.sqrt((J * J).sum(axis=0))[None, :]


def measurements(J32: np.ndarray, truth: np.ndarray, seed: int, snr_db: float = 40.0,
                 stream_offset: int = 0, Jn: np.ndarray | None = None) -> np.ndarray:
    """Delta v for each truth frame: J_n @ truth_t + noise (float32, shape (T, M)).

    ``truth`` is (T, V).  The noise standard deviation is 10^(-snr/20) times the RMS of the
    clean measurement of the peak-amplitude frame, held fixed across frames; noise is drawn
    i.i.d. per frame and measurement.
    """
    truth = np.atleast_2d(truth)
    if Jn is None:
        Jn = column_normalised(J32)
    clean = truth @ Jn.T                                   # (T, M)
    peak = int(np.argmax(np.abs(truth).sum(axis=1)))
    rms = math.sqrt(float(np.mean(clean[peak] ** 2)))
    sd = 10.0 ** (-snr_db / 20.0) * rms
    T, M = clean.shape
    noise = normal(seed, STREAM_NOISE, T * M, offset=stream_offset).reshape(T, M)
    return (clean + sd * noise).astype(np.float32)


def input_noise(n: int, channels: int, seed: int, std: float = 0.1,
                stream_offset: int = 0) -> np.ndarray:
    """Fixed network input Z: N(0, std^2), float32, shape (n, channels) (channels fastest)."""
    return (std * normal(seed, STREAM_Z, n * channels, offset=stream_offset)).reshape(
        n, channels).astype(np.float32)


# --------------------------------------------------------------------------------------
# Initial weights
# --------------------------------------------------------------------------------------

KIND_CONV_W = 0
KIND_CONV_B = 1
KIND_LN_G = 2
KIND_LN_B = 3


def kaiming_theta(table, seed: int, stream_offset: int = 0) -> np.ndarray:
    """Kaiming-normal initial weights for a flat parameter arena.

    ``table`` is a sequence of (kind, offset, count, fan_in) rows.  Conv weights get
    N(0, 2/fan_in) (He et al., gain sqrt(2)); conv biases and LayerNorm shifts 0; LayerNorm
    scales 1.  Returns float32 of length max(offset+count).
    """
    size = max(int(o) + int(c) for _, o, c, _ in table)
    theta = np.zeros(size, dtype=np.float64)
    for idx, (kind, off, cnt, fan_in) in enumerate(table):
        off, cnt = int(off), int(cnt)
        if kind == KIND_CONV_W:
            std = math.sqrt(2.0 / float(fan_in))
            theta[off:off + cnt] = std * normal(seed, STREAM_THETA, cnt,
                                                offset=stream_offset + off)
        elif kind == KIND_LN_G:
            theta[off:off + cnt] = 1.0
        elif kind in (KIND_CONV_B, KIND_LN_B):
            theta[off:off + cnt] = 0.0
        else:
            raise ValueError(f"unknown parameter kind {kind} in row {idx}")
    return theta.astype(np.float32)


# --------------------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    grid: tuple[int, int, int]
    rings: int
    levels: int
    widths: tuple[int, ...]
    c_in: int
    frames: int
    upws_steps: int
    first_steps: int
    later_steps: int
    lr: float
    seed: int

    @property
    def n(self) -> int:
        X, Y, Z = self.grid
        return X * Y * Z

    @property
    def m(self) -> int:
        return self.rings * MEAS_PER_RING


# plain single-frame DIP: 16x16x8, one ring, 2 levels 8/16, 200 steps, lr 1e-3
SINGLE_16 = Workload("single-frame 16x16x8 m208 L2(8,16)", (16, 16, 8), 1, 2, (8, 16), 8,
                     1, 0, 200, 200, 1e-3, 0)
# 20-frame breathing sequence: 32x32x16, two rings, 3 levels 16/32/64, 300 UPWS + 50/frame
SEQ_32 = Workload("20-frame sequence 32x32x16 m416 L3(16,32,64)", (32, 32, 16), 2, 3,
                  (16, 32, 64), 8, 20, 300, 50, 50, 5e-4, 0)
# 100-frame breathing sequence: 64x64x32, three rings, 4 levels 16..128, 400 UPWS + 40/frame
SEQ_64 = Workload("100-frame sequence 64x64x32 m624 L4(16,32,64,128)", (64, 64, 32), 3, 4,
                  (16, 32, 64, 128), 8, 100, 400, 40, 40, 5e-4, 0)


def sequence_truth(w: Workload) -> np.ndarray:
    """(T, V) truth: the lung pair at -0.3 * breathing amplitude (single frame: amplitude 1)."""
    base = ellipsoid_phantom(w.grid, lung_pair(w.grid), -0.3)
    if w.frames == 1:
        return base[None, :]
    return breathing_amplitude(w.frames)[:, None] * base[None, :]


def make_problem(w: Workload):
    """Raw J (float32), truth (float64, T x V), measurements (float32, T x M), Z (float32)."""
    J = sensitivity_raw(w.grid, w.rings, w.seed)
    truth = sequence_truth(w)
    V = measurements(J, truth, w.seed)
    Zin = input_noise(w.n, w.c_in, w.seed)
    return J, truth, V, Zin


BATCH_GRIDS = ((16, 16, 8), (32, 32, 16), (48, 48, 24))
BATCH_RINGS = (1, 2)


def batch_problem_shapes(count: int, seed: int) -> list[tuple[tuple[int, int, int], int]]:
    """(grid, rings) for each of ``count`` independent sequences: grid uniform over
    16x16x8 / 32x32x16 / 48x48x24 and m uniform over {208, 416}."""
    u = uniform(seed, STREAM_BATCH, 2 * count)
    out = []
    for p in range(count):
        g = BATCH_GRIDS[min(2, int(u[2 * p] * 3))]
        r = BATCH_RINGS[min(1, int(u[2 * p + 1] * 2))]
        out.append((g, r))
    return out


@dataclass
class BatchGroup:
    """Problems of the batched workload that share a grid and a measurement count (hence one
    sensitivity matrix)."""
    grid: tuple[int, int, int]
    rings: int
    J: np.ndarray                 # raw float32 (m, n)
    problems: list[int]           # indices into the 64 sequences
    truth: np.ndarray             # (B, T, n) float64
    V: np.ndarray                 # (B, T, m) float32
    Z: np.ndarray                 # (B, n, c_in) float32


def batch_sensitivity_seed(grid, rings, seed: int = 1) -> int:
    """J depends only on (grid, m), seeded from (seed, X, Y, Z, m)."""
    X, Y, Z = grid
    k = _key(seed, ((X * 1009 + Y) * 1013 + Z) * 4099 + rings * MEAS_PER_RING)
    return int(k & np.uint64(0x7FFFFFFF))


def batch_workload(count: int = 64, frames: int = 20, seed: int = 1, c_in: int = 8):
    """The batched workload: ``count`` independent breathing sequences on random grids and
    electrode counts with random ellipsoid pairs, grouped by (grid, rings)."""
    shapes = batch_problem_shapes(count, seed)
    keys = sorted(set(shapes), key=lambda k: (k[0][0], k[1]))
    amp = breathing_amplitude(frames)
    groups = []
    for g, r in keys:
        idx = [p for p, sh in enumerate(shapes) if sh == (g, r)]
        J = sensitivity_raw(g, r, batch_sensitivity_seed(g, r, seed))
        Jn = column_normalised(J)
        n = g[0] * g[1] * g[2]
        truths, Vs, Zs = [], [], []
        for p in idx:
            base = ellipsoid_phantom(g, random_ellipsoids(g, seed, p), -0.3)
            t = amp[:, None] * base[None, :]
            truths.append(t)
            Vs.append(measurements(J, t, seed, stream_offset=p * 1_000_003, Jn=Jn))
            Zs.append(input_noise(n, c_in, seed, stream_offset=p * 10_000_019))
        groups.append(BatchGroup(g, r, J, idx, np.stack(truths), np.stack(Vs), np.stack(Zs)))
    return groups
