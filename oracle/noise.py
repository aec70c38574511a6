"""Z(4) noise vectors (Sec. 1: eta with components in Z(4); "unpartitioned",
i.e. full volume and all spin-colour components, Sec. 4).

Reading taken (the paper does not fix the generator): component values are
i^code, code in {0, 1, 2, 3}, i.e. {1, i, -1, -i} with equal probability.
For site s (lexicographic, x fastest), noise index j, level id l and stream
tag g, one Philox4x32-10 call with counter (s, j, l, g) and key
(seed mod 2^32, seed >> 32) gives word w0; spin-colour component
c = 3*spin + colour takes code (w0 >> 2c) & 3.
"""
import numpy as np

from .philox import philox4x32_10

TAG_NOISE = 0x4E4F4953   # 'NOIS'
TAG_GMRES = 0x474D5253   # 'GMRS'
TAG_ARNOLDI = 0x4445464C  # 'DEFL'

_Z4 = np.array([1, 1j, -1, -1j], dtype=np.complex128)


def z4_codes(dims, seed, noise_index, level_id, tag=TAG_NOISE):
    """Integer codes, shape [t][z][y][x][4][3], for one noise vector."""
    lx, ly, lz, lt = dims
    vol = lx * ly * lz * lt
    site = np.arange(vol, dtype=np.uint64)
    w0, _, _, _ = philox4x32_10(site, noise_index, level_id, tag, seed & 0xFFFFFFFF, seed >> 32)
    shifts = 2 * np.arange(12, dtype=np.uint32)
    codes = (w0[:, None] >> shifts[None, :]) & np.uint32(3)
    return codes.reshape(lt, lz, ly, lx, 4, 3).astype(np.int64)


def z4_noise(dims, seed, noise_index, level_id, tag=TAG_NOISE):
    """One Z(4) noise vector in canonical layout [t][z][y][x][spin][colour]."""
    return _Z4[z4_codes(dims, seed, noise_index, level_id, tag)]


def z4_noise_batch(dims, seed, noise_indices, level_id, tag=TAG_NOISE):
    """Noise vectors for several indices, stacked on a trailing batch axis."""
    return np.stack([z4_noise(dims, seed, j, level_id, tag) for j in noise_indices], axis=-1)
