"""The gather's shared-memory bands hold every pair its pixels read (CPU).

The gather stages, per angle, a band of kBand sinogram pair slots starting at
the slot of the tile origin's projection plus floor(31 min(cos, 0)) - 1,
rounded down to a 16-byte boundary; a pixel then reads pair slot p >> 23 of
the band (one element holding the two bins the pixel meets), with p its 9.23
fixed-point position (the origin's fraction plus integer multiples of cos and
sin in 9.23).  Every read must satisfy 0 <= p >> 23 < kBand, or it would leave
the band.

This recomputes, with the same fixed-point steps, the smallest and largest
band index of every tile, angle (slot) and position window of the
mirror-paired path (32 x 16 tiles of the left half; windows at the angle and
at its mirror, cos -> -cos) for every image size the batch and the server
draw, and of the plain path's 32 x 32 tiles, on the angle table of the
library (angles past pi/2 through cos(pi - t) = -cos t).
"""
import math

import numpy as np
import pytest

K_SPAD = 2                     # zero pairs before each sinogram-view row
TWO32 = 2.0 ** 32
TWO23 = 2.0 ** 23


def angle_table(na):
    """cos, sin of theta_a = pi a / na, exact mirrors past pi/2 (as the library's table)."""
    c = np.empty(na)
    s = np.empty(na)
    for a in range(na):
        if a == 0:
            c[a], s[a] = 1.0, 0.0
        elif 2 * a == na:
            c[a], s[a] = 0.0, 1.0
        else:
            mirror = 2 * a > na
            th = math.pi * (na - a if mirror else a) / na
            c[a] = -math.cos(th) if mirror else math.cos(th)
            s[a] = math.sin(th)
    return c, s


def band_extremes(n, na, nb, tile_h, windows, slots_per_seg):
    """Smallest and largest band index over all tiles, angles and windows."""
    c, s = angle_table(na)
    c_fx = np.rint(c * TWO32).astype(np.int64)
    s_fx = np.rint(s * TWO32).astype(np.int64)
    c23 = np.rint(c * TWO23).astype(np.int64)
    s23 = np.rint(s * TWO23).astype(np.int64)
    cols = n // 2 if windows == 2 else n          # mirror path: the left half's tiles
    j0 = np.arange(0, cols, 32)
    i0 = np.arange(0, n, tile_h)
    X2 = (2 * j0 - (n - 1))[:, None, None]
    Y2 = (2 * i0 - (n - 1))[None, :, None]
    lo_idx, hi_idx = 10 ** 9, -10 ** 9
    for w in range(windows):
        sign = -1 if w == 1 else 1                # window B: T at the mirror of the angle
        cf = sign * c_fx[None, None, :]
        cb = ((nb - 1) << 31) + ((X2 * cf + Y2 * s_fx[None, None, :]) >> 1)
        cw = (sign * c).astype(np.float32)
        lo = np.floor(np.float32(31) * np.minimum(cw, np.float32(0))).astype(np.int64) - 1
        I = cb >> 32
        s_lo = (I + K_SPAD + lo[None, None, :]) & ~(slots_per_seg - 1)
        base = ((I + K_SPAD - s_lo) << 23) | ((cb & 0xFFFFFFFF) >> 9)
        dc = sign * c23[None, None, :]
        p_min = base + np.minimum(0, 31 * dc) + np.minimum(0, (tile_h - 1) * s23[None, None, :])
        p_max = base + np.maximum(0, 31 * dc) + np.maximum(0, (tile_h - 1) * s23[None, None, :])
        assert p_min.min() >= 0
        lo_idx = min(lo_idx, int((p_min >> 23).min()))
        hi_idx = max(hi_idx, int((p_max >> 23).max()))
    return lo_idx, hi_idx


def bins_for(n):
    return int(math.ceil(math.sqrt(2.0) * n))


BATCH = [(n, na) for n in (128, 192, 256, 384, 512, 768) for na in (60, 120, 180, 360, 720)]
SERVING = [(n, na) for n in range(128, 1025, 64) for na in (30, 31, 90, 180)]
SINGLE = [(512, 720), (1024, 1440), (64, 90), (64, 1), (64, 2), (64, 7)]


@pytest.mark.parametrize("n,na", BATCH + SERVING + SINGLE)
def test_mirror_path_bands_hold_every_pair(n, na):
    nb = 725 if (n, na) == (512, 720) else 1449 if (n, na) == (1024, 1440) else bins_for(n)
    for k_band, per_seg in ((48, 2), (52, 4)):    # FP32 pairs, 16-bit pairs
        lo, hi = band_extremes(n, na, nb, 16, 2, per_seg)
        # the 32 x 16 tiles need at most 31 |c| + 15 s + 4 < 40 slots of the 48 (52)
        assert lo >= 0 and hi <= 40, (n, na, k_band, lo, hi)


@pytest.mark.parametrize("n,na,nb", [(512, 720, 725), (77, 33, 110), (130, 181, 185), (33, 4, 47), (2, 3, 3)])
def test_plain_path_bands_hold_every_pair(n, na, nb):
    # 32 x 32 tiles: at most 31 (|c| + s) + 4 < 48 slots (47.8 at 45 degrees)
    for k_band, per_seg in ((48, 2), (52, 4)):
        lo, hi = band_extremes(n, na, nb, 32, 1, per_seg)
        assert lo >= 0 and hi <= k_band - 1, (n, na, k_band, lo, hi)
