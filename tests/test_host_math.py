"""Arithmetic facts the kernels rely on, checked on the CPU.

The tube tile computes j div nf (and j mod nf) for the mode-3 length nf <= 8 as
floor(j * ceil(2^16 / nf) / 2^16); the tile form's indices stay below nf * nh <= 8 * 254 (tube
offsets, hh = nh / 2 + 1 <= 128) and nf * hh <= 8 * 128 (spectrum rows).  The identity must be
exact over that whole range (it holds up to 8191 for every nf <= 8)."""


def _div(j, nf):
    m = (65536 + nf - 1) // nf
    return (j * m) >> 16


def test_reciprocal_division_is_exact_over_the_tile_indices():
    for nf in range(1, 9):
        for j in range(8192):
            assert _div(j, nf) == j // nf, (nf, j)
    # the largest tile-form index is well inside that range
    assert 8 * 254 < 8192 and 8 * 128 < 8192
