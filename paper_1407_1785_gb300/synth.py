"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

Nothing here belongs to the t-SVT / ADMM arithmetic: this module only draws random numbers
and assembles test tensors.  Both the CUDA library and the FP64 oracle consume its arrays as
plain inputs, so neither side generates its own data.

Random numbers come from a counter-based SplitMix64: for a (seed, stream) pair the key is
``mix64(seed ^ (stream << 56))`` and draw ``i`` is ``mix64(key + (i + 1) * GAMMA)``, where
``mix64`` is SplitMix64's output function and ``GAMMA = 0x9E3779B97F4A7C15`` its increment.
So every draw depends only on (seed, stream, index), whatever the array shape or platform.

  uniform in [0, 1)  : (h >> 11) * 2**-53
  Bernoulli(p)       : (h >> 11) < floor(p * 2**53)          (integer compare, bit-exact)
  standard normal    : Box-Muller on draws 2i, 2i+1 in FP64

Streams: 0 = factor A, 1 = factor B, 2 = sampling mask Omega, 3 = sparse support,
4 = sparse values, 5 = additive noise, 6 = texture parameters, 7 = batch shapes.

Array convention: numpy arrays of shape (n1, n2, n3[, n4]); the library and the oracle take
them in MATLAB column-major order (``to_colmajor`` / ``from_colmajor``).

The synthetic workloads stand in for the paper's videos (Escalator, MERL and Basketball,
Sec. 3 / Sec. 4 / Sec. 5), which are not available: a low-tubal-rank t-product, a smooth
texture translating under linear camera motion (the panning-camera case of Sec. 3), and
sparse entrywise or tube-wise corruptions (Sec. 5).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_A, STREAM_B, STREAM_OMEGA, STREAM_SUPPORT, STREAM_SVALUES = 0, 1, 2, 3, 4
STREAM_NOISE, STREAM_TEXTURE, STREAM_BATCH = 5, 6, 7


def _mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def hash64(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """64-bit counter-based draws for indices `index` of (seed, stream)."""
    key = _mix64(np.uint64((int(seed) ^ (int(stream) << 56)) & 0xFFFFFFFFFFFFFFFF))
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(key + (idx + np.uint64(1)) * GAMMA)


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    h = hash64(seed, stream, np.arange(offset, offset + n, dtype=np.uint64))
    return (h >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def bernoulli(seed: int, stream: int, n: int, p: float) -> np.ndarray:
    """uint8 0/1 draws with P(1) = p, decided by an integer compare."""
    h = hash64(seed, stream, np.arange(n, dtype=np.uint64))
    thresh = np.uint64(int(math.floor(float(p) * 2.0 ** 53)))
    return ((h >> np.uint64(11)) < thresh).astype(np.uint8)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """Standard normals by Box-Muller; output i uses draws 2i and 2i+1."""
    m = (n + 1) // 2
    u = uniform(seed, stream, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))          # 1 - u1 is in (0, 1]
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:n]


def to_colmajor(x: np.ndarray, dtype=np.float32) -> np.ndarray:
    """Flatten an (n1, n2, ...) array in MATLAB column-major order."""
    return np.asfortranarray(np.asarray(x, dtype=dtype)).ravel(order="F").copy()


def from_colmajor(v: np.ndarray, shape) -> np.ndarray:
    return np.reshape(np.asarray(v), tuple(shape), order="F")


def _normal_tensor(seed: int, stream: int, shape) -> np.ndarray:
    n = int(np.prod(shape))
    return from_colmajor(normal(seed, stream, n), shape)


def circular_tproduct(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """t-product by its definition (Def. 2.1.1): tube (i,j) of C is the sum over k of the
    circular convolutions A(i,k,:) o B(k,j,:).  Written as n3 shifted slice products:
    C(:,:,t) = sum_s A(:,:,s) @ B(:,:,(t - s) mod n3)."""
    n1, n2, n3 = A.shape
    n2b, n4, n3b = B.shape
    assert n2 == n2b and n3 == n3b
    C = np.zeros((n1, n4, n3))
    for t in range(n3):
        for s in range(n3):
            C[:, :, t] += A[:, :, s] @ B[:, :, (t - s) % n3]
    return C


def lowrank_tensor(n1: int, n2: int, n3: int, rank: int, seed: int):
    """X = A * B with A (n1 x rank x n3), B (rank x n2 x n3) iid N(0,1): tubal rank <= rank."""
    A = _normal_tensor(seed, STREAM_A, (n1, rank, n3))
    B = _normal_tensor(seed, STREAM_B, (rank, n2, n3))
    return circular_tproduct(A, B)


def sampling_mask(shape, p: float, seed: int) -> np.ndarray:
    """Omega: each entry observed independently with probability p (uint8 0/1)."""
    n = int(np.prod(shape))
    return from_colmajor(bernoulli(seed, STREAM_OMEGA, n, p), shape)


def translating_texture(n1: int, n2: int, n3: int, seed: int, n_bumps: int = 20,
                        shift=(0.7, 0.4), noise_std: float = 0.01, channel: int = 0):
    """A smooth random texture under linear camera motion, one frame per slice.

    The texture is a sum of `n_bumps` 2-D Gaussian bumps on a canvas of
    (n1 + ceil(0.7 n3) + 2) x (n2 + ceil(0.4 n3) + 2) pixels (centres uniform on the canvas,
    widths uniform in [4, 16] px, amplitudes uniform in [0.2, 1]), min-max normalised to
    [0, 1].  Frame t samples it bilinearly at (i + 0.7 t, j + 0.4 t); then N(0, noise_std^2)
    noise is added.  `channel` selects an independent texture (and noise) per colour channel.
    """
    dr, dc = shift
    H = n1 + int(math.ceil(dr * n3)) + 2
    W = n2 + int(math.ceil(dc * n3)) + 2
    par = uniform(seed, STREAM_TEXTURE, 5 * n_bumps, offset=5 * n_bumps * channel)
    par = par.reshape(n_bumps, 5)
    cy, cx = par[:, 0] * H, par[:, 1] * W
    sig = 4.0 + 12.0 * par[:, 2]
    amp = 0.2 + 0.8 * par[:, 3]
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                         indexing="ij")
    tex = np.zeros((H, W))
    for b in range(n_bumps):
        tex += amp[b] * np.exp(-((yy - cy[b]) ** 2 + (xx - cx[b]) ** 2) / (2.0 * sig[b] ** 2))
    tex = (tex - tex.min()) / max(tex.max() - tex.min(), 1e-300)
    ii, jj = np.meshgrid(np.arange(n1, dtype=np.float64), np.arange(n2, dtype=np.float64),
                         indexing="ij")
    out = np.empty((n1, n2, n3))
    for t in range(n3):
        y = ii + dr * t
        x = jj + dc * t
        y0 = np.floor(y).astype(np.int64)
        x0 = np.floor(x).astype(np.int64)
        fy, fx = y - y0, x - x0
        out[:, :, t] = ((1 - fy) * (1 - fx) * tex[y0, x0] + (1 - fy) * fx * tex[y0, x0 + 1]
                        + fy * (1 - fx) * tex[y0 + 1, x0] + fy * fx * tex[y0 + 1, x0 + 1])
    n = n1 * n2 * n3
    noise = normal(seed, STREAM_NOISE, n * (channel + 1))[n * channel:]
    return out + noise_std * from_colmajor(noise, (n1, n2, n3))


def sparse_corruption(shape, frac: float, seed: int, lo: float = -5.0, hi: float = 5.0):
    """Entrywise sparse tensor: support ~ Bernoulli(frac), values uniform in [lo, hi]."""
    n = int(np.prod(shape))
    sup = bernoulli(seed, STREAM_SUPPORT, n, frac)
    val = lo + (hi - lo) * uniform(seed, STREAM_SVALUES, n)
    return from_colmajor(sup * val, shape), from_colmajor(sup, shape)


def tube_corruption(shape, frac: float, seed: int, block: int = 10, std: float = 1.0):
    """Tube-wise sparse noise as in the tensor RPCA experiment of Sec. 5: a fraction `frac`
    of pixel tubes carry Gaussian noise, and the noisy pixel locations stay the same within
    each block of `block` consecutive frames."""
    n1, n2, n3 = shape
    nblk = (n3 + block - 1) // block
    sup_blocks = from_colmajor(bernoulli(seed, STREAM_SUPPORT, n1 * n2 * nblk, frac),
                               (n1, n2, nblk))
    sup = np.repeat(sup_blocks, block, axis=2)[:, :, :n3]
    val = std * from_colmajor(normal(seed, STREAM_SVALUES, n1 * n2 * n3), shape)
    return sup * val, sup.astype(np.uint8)


# ---------------------------------------------------------------------------------------------
# The workloads (shapes, sampling rates and corruption levels used in tests and benches).
# ---------------------------------------------------------------------------------------------

def workload_lowrank_completion(seed: int = 1, n1=32, n2=32, n3=16, rank=3, p=0.5):
    """Low-tubal-rank completion: X = A*B (rank 3, 32x32x16), 50% of entries observed."""
    X = lowrank_tensor(n1, n2, n3, rank, seed)
    omega = sampling_mask(X.shape, p, seed)
    return X, omega


def workload_video_completion(seed: int = 1, n1=144, n2=176, n3=100, p=0.2):
    """Grayscale video completion: 144x176x100 translating texture + N(0, 0.01^2) noise,
    20% of entries observed uniformly at random."""
    X = translating_texture(n1, n2, n3, seed)
    omega = sampling_mask(X.shape, p, seed)
    return X, omega


def workload_rpca(seed: int = 1, n1=240, n2=320, n3=60, rank=10, frac=0.1):
    """Tensor RPCA: L tubal rank 10 (240x320x60), S = 10% entries uniform in [-5, 5],
    lambda = 1/sqrt(max(n1, n2) n3)."""
    L = lowrank_tensor(n1, n2, n3, rank, seed)
    S, sup = sparse_corruption(L.shape, frac, seed)
    lam = 1.0 / math.sqrt(max(n1, n2) * n3)
    return L + S, L, S, sup, lam


def workload_rpca_tube(seed: int = 1, n1=144, n2=256, n3=80, frac=0.1, block=10, std=1.0):
    """Tube-sparse tensor RPCA on video (the Sec. 5 experiment's setting, at the size of its
    144 x 256 x 80 clip): L = a panning-texture video, S = Gaussian noise (std 1) on a fraction
    `frac` of the pixel tubes, the noisy pixels fixed within each block of `block` frames;
    lambda = 1/sqrt(max(n1, n2)) for the l_{1,1,2} term of eq. sparse2."""
    L = translating_texture(n1, n2, n3, seed)
    S, sup = tube_corruption(L.shape, frac, seed, block=block, std=std)
    lam = 1.0 / math.sqrt(max(n1, n2))
    return L + S, L, S, sup, lam


def workload_color_video(seed: int = 1, n1=288, n2=352, n3=3, n4=60, p=0.15):
    """4-way colour video completion: 288x352x3x60, an independent translating texture per
    channel, 15% of entries observed."""
    X = np.empty((n1, n2, n3, n4))
    for c in range(n3):
        X[:, :, c, :] = translating_texture(n1, n2, n4, seed, channel=c)
    omega = sampling_mask(X.shape, p, seed)
    return X, omega


def workload_multiview_video(seed: int = 1, n1=144, n2=176, nc=3, nv=2, nt=40, p=0.2):
    """5-way multi-view colour video completion: 144x176 frames x 3 channels x 2 views x 40
    frames, an independent translating texture per (channel, view), 20% of entries observed.
    The t-SVD takes the DFT along modes 3, 4 and 5."""
    X = np.empty((n1, n2, nc, nv, nt))
    for v in range(nv):
        for c in range(nc):
            X[:, :, c, v, :] = translating_texture(n1, n2, nt, seed, channel=c + nc * v)
    omega = sampling_mask(X.shape, p, seed)
    return X, omega


def workload_batch_shapes(seed: int = 1, count: int = 64):
    """Shapes of the uneven batch: n1, n2 uniform in [48, 256], n3 uniform in [8, 64],
    tubal rank uniform in [2, 12]; even index -> completion with observed fraction in
    [0.2, 0.6], odd index -> RPCA with corruption fraction in [0.05, 0.15]."""
    u = uniform(seed, STREAM_BATCH, 5 * count).reshape(count, 5)
    out = []
    for b in range(count):
        n1 = 48 + int(u[b, 0] * 209)
        n2 = 48 + int(u[b, 1] * 209)
        n3 = 8 + int(u[b, 2] * 57)
        rank = 2 + int(u[b, 3] * 11)
        if b % 2 == 0:
            out.append(dict(kind="complete", n1=n1, n2=n2, n3=n3, rank=rank,
                            p=0.2 + 0.4 * u[b, 4]))
        else:
            out.append(dict(kind="rpca", n1=n1, n2=n2, n3=n3, rank=rank,
                            frac=0.05 + 0.10 * u[b, 4]))
    return out


def workload_batch(seed: int = 1, count: int = 64):
    """The uneven batch itself: for tensor b of `workload_batch_shapes`, with per-tensor seed
    s = 1000 seed + b, L = a tubal-rank-r t-product of N(0,1) factors; completion tensors
    observe L on Omega ~ Bernoulli(p); RPCA tensors see M = L + S with S an entrywise
    corruption (fraction `frac`, values uniform in [-5, 5]) and lambda = 1/sqrt(max(n1, n2) n3).
    Returns a list of dicts with kind, dims, M (float32, Omega-projected for completion),
    omega (completion) or lam (RPCA), and truth (the float64 L)."""
    items = []
    for b, sp in enumerate(workload_batch_shapes(seed=seed, count=count)):
        s = seed * 1000 + b
        L = lowrank_tensor(sp["n1"], sp["n2"], sp["n3"], sp["rank"], seed=s)
        if sp["kind"] == "complete":
            om = sampling_mask(L.shape, sp["p"], seed=s)
            items.append(dict(kind="complete", dims=L.shape, M=(L * om).astype(np.float32),
                              omega=om, truth=L))
        else:
            S, _ = sparse_corruption(L.shape, sp["frac"], seed=s)
            lam = 1.0 / math.sqrt(max(sp["n1"], sp["n2"]) * sp["n3"])
            items.append(dict(kind="rpca", dims=L.shape, M=(L + S).astype(np.float32),
                              lam=lam, truth=L))
    return items


def sample_indices(n: int, k: int, seed: int = 20260101) -> np.ndarray:
    """k distinct flat (column-major) indices of an n-entry tensor, sorted, drawn from the
    counter-based generator (the first k distinct values of floor(u n) in draw order): where
    stored expected values are a sample of a large output."""
    k = min(k, n)
    draws = 4 * k + 64
    while True:
        v = (uniform(seed, STREAM_BATCH + 1, draws) * n).astype(np.int64)
        _, first = np.unique(v, return_index=True)
        if first.size >= k:
            return np.sort(v[np.sort(first)[:k]])
        draws *= 2
