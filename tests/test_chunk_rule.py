"""The z-chunk of sweep launches over fewer than six load cases
(ce_sweep_chunk, host logic, no GPU): the choices measured fastest at 191^3,
the tile's chunk where waves are many or the rule does not apply, and the
bound that keeps every launch's residual partials inside the buffer sized
for the tile."""
import math

import pytest

from paper_2410_20441_gb300 import ce


def test_measured_choices_at_191():
    # 24-row blocks, 96-plane chunks, 152 SMs: the correction-phase launch
    # times measured on a GB300 were fastest at 32, 48, 64 and 48 planes for
    # 2, 3, 4 and 5 cases; one case and six keep the tile's chunk
    got = [ce.sweep_chunk((191, 191, 191), (3, 24, 96, 1), n, 152) for n in range(1, 7)]
    assert got == [96, 32, 48, 64, 48, 96]


def test_many_waves_keep_the_tile_chunk():
    assert {ce.sweep_chunk((479, 479, 479), (3, 24, 48, 1), n, 152) for n in range(1, 7)} == {48}
    assert {ce.sweep_chunk((703, 703, 703), (3, 24, 48, 1), n, 152) for n in range(1, 7)} == {48}


def test_rule_off_for_paired_columns_or_unknown_sms():
    assert ce.sweep_chunk((191, 191, 191), (3, 8, 24, 2), 2, 152) == 24
    assert ce.sweep_chunk((191, 191, 191), (3, 24, 96, 1), 3, 0) == 96
    assert ce.sweep_chunk((191, 191, 191), (0, 0, 0, 0), 6, 152) == 32   # the default chunk


@pytest.mark.parametrize("shape,tile", [((191, 191, 191), (3, 24, 96, 1)), ((64, 40, 90), (3, 16, 0, 1)),
                                        ((127, 127, 127), (2, 8, 48, 1)), ((31, 33, 29), (3, 16, 256, 1)),
                                        ((300, 100, 60), (3, 24, 16, 1))])
def test_partials_bound_and_chunk_floor(shape, tile):
    nz = shape[0]
    span = nz + 1
    zc0 = tile[2] if tile[2] > 0 else 32
    nch0 = math.ceil(span / zc0)
    for nsm in (16, 152):
        for n in range(1, 7):
            zc = ce.sweep_chunk(shape, tile, n, nsm)
            assert zc == zc0 or zc >= 16
            # residual partials: n cases x chunks fit in 6 x (2 nch0 + 1) chunks' room
            assert n * math.ceil(span / zc) <= 6 * (2 * nch0 + 1)


def test_bad_arguments_are_rejected():
    with pytest.raises(ce.CeError):
        ce.sweep_chunk((191, 191, 191), (3, 24, 96, 1), 0, 152)
    with pytest.raises(ce.CeError):
        ce.sweep_chunk((191, 191, 191), (3, 24, 96, 1), 7, 152)
    with pytest.raises(ce.CeError):
        ce.sweep_chunk((1, 191, 191), (3, 24, 96, 1), 3, 152)
