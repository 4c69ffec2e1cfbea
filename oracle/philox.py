"""Counter-based random numbers for the stochastic stress (oracle side).

The paper draws the stochastic stress from white noise W with unit covariance
per cell and per step, combined across the three Runge-Kutta stages as
W_1 = W_A - sqrt(3) W_B, W_2 = W_A + sqrt(3) W_B, W_3 = W_A (App. A.2).  It
does not name a generator.  Both sides of this project use Philox4x32-10
(Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11), written here from its published definition, so that every draw is a
pure function of (seed, box, cell, step, purpose, block) and can be reproduced
bit for bit on the GPU.

Stream map (shared by specification, not by code, with the CUDA library)
----------------------------------------------------------------------
key     = (seed & 0xffffffff, seed >> 32)
counter = (cell, step, (purpose << 16) | block, box)

purpose 0 (stochastic stress): blocks 0..5 give 24 words per cell and step.
    Normal j (j = 0..11; 0..5 are stream A components xx, yy, zz, xy, xz, yz,
    6..11 the same components of stream B) takes its high word from word j
    and its low word from word 12 + j.
purpose 1 (thermal initial state): blocks 0..1 give 8 words per cell; normals
    j = 0..3 (delta rho, g_x, g_y, g_z) take high word j, low word 4 + j.

A 52-bit uniform is u = (2 m + 1) 2^-53 with m = (hi << 20) | (lo >> 12), which
lies strictly inside (0, 1) and is exact in binary64.  Normals come in
Box-Muller pairs (n_{2i}, n_{2i+1}) = r (cos 2 pi u_{2i+1}, sin 2 pi u_{2i+1}),
r = sqrt(-2 ln u_{2i}) (Box and Muller, 1958).
"""
import numpy as np

PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)

PURPOSE_STRESS = 0
PURPOSE_THERMAL = 1


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds.

    ctr : uint32 array of shape (..., 4); key : uint32 array of shape (..., 2)
    (broadcast against ctr).  Returns uint32 array of shape (..., 4).

    One round maps (c0, c1, c2, c3) with key (k0, k1) to
    (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0));
    the key is bumped by the Weyl constants (W0, W1) between rounds.
    """
    c = np.asarray(ctr, dtype=np.uint32).astype(np.uint64)
    k = np.asarray(key, dtype=np.uint32).astype(np.uint64)
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0 = np.broadcast_to(k[..., 0], c0.shape).copy()
    k1 = np.broadcast_to(k[..., 1], c0.shape).copy()
    for r in range(10):
        p0 = PHILOX_M0 * c0          # exact: both factors < 2^32
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if r < 9:
            k0 = (k0 + np.uint64(PHILOX_W0)) & MASK32
            k1 = (k1 + np.uint64(PHILOX_W1)) & MASK32
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def seed_key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)


def words(seed, box, cells, step, purpose, nblocks):
    """Raw words for each cell: uint32 array (ncells, 4 * nblocks)."""
    cells = np.asarray(cells, dtype=np.uint64).astype(np.uint32)
    n = cells.shape[0]
    out = np.empty((n, 4 * nblocks), dtype=np.uint32)
    key = seed_key(seed)
    for b in range(nblocks):
        ctr = np.empty((n, 4), dtype=np.uint32)
        ctr[:, 0] = cells
        ctr[:, 1] = np.uint32(int(step) & 0xFFFFFFFF)
        ctr[:, 2] = np.uint32(((int(purpose) & 0xFFFF) << 16) | b)
        ctr[:, 3] = np.uint32(int(box) & 0xFFFFFFFF)
        out[:, 4 * b:4 * b + 4] = philox4x32_10(ctr, key)
    return out


def uniform52(hi, lo):
    """u = (2 m + 1) 2^-53, m = (hi << 20) | (lo >> 12): strictly in (0, 1)."""
    m = (hi.astype(np.uint64) << np.uint64(20)) | (lo.astype(np.uint64) >> np.uint64(12))
    return (2.0 * m.astype(np.float64) + 1.0) * 2.0 ** -53


def box_muller(u):
    """Pairs of uniforms (rows 2i, 2i+1) -> pairs of standard normals."""
    n = np.empty_like(u)
    for i in range(u.shape[0] // 2):
        r = np.sqrt(-2.0 * np.log(u[2 * i]))
        th = 2.0 * np.pi * u[2 * i + 1]
        n[2 * i] = r * np.cos(th)
        n[2 * i + 1] = r * np.sin(th)
    return n


def stress_normals(seed, box, step, ncells):
    """The 12 unit normals per cell for one step: array (12, ncells).

    Rows 0..5 are W_A (xx, yy, zz, xy, xz, yz), rows 6..11 are W_B.
    """
    return stress_normals_at(seed, box, step, np.arange(ncells))


def stress_normals_at(seed, box, step, cells):
    """The same 12 normals for the given linear cell indices only: (12, len(cells))."""
    w = words(seed, box, cells, step, PURPOSE_STRESS, 6)
    u = uniform52(w[:, 0:12].T, w[:, 12:24].T)
    return box_muller(u)


def thermal_normals(seed, box, ncells):
    """The 4 unit normals per cell for the thermal initial state: (4, ncells)."""
    w = words(seed, box, np.arange(ncells), 0, PURPOSE_THERMAL, 2)
    u = uniform52(w[:, 0:4].T, w[:, 4:8].T)
    return box_muller(u)
