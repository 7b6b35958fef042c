"""Host logic of the c-transform shape tuner (no GPU): the candidate shapes
of each kernel kind and line length are valid launch shapes and include the
hand-picked default, the shape table stores and forgets shapes, and the
pick keeps the default unless a candidate beats it by the margin."""
import pytest

from paper_1905_12154_gb300 import binding as B

KINDS = (B.CT_KIND_TILE_ROWS, B.CT_KIND_TILE_COLS, B.CT_KIND_ROW, B.CT_KIND_ROW_COLS)
ROW_KINDS = (B.CT_KIND_ROW, B.CT_KIND_ROW_COLS)


def _next_pow2(x):
    p = 1
    while p < x:
        p *= 2
    return p


@pytest.fixture(autouse=True)
def clean_table():
    B.bfm_tune_clear()
    yield
    B.bfm_tune_clear()


@pytest.mark.parametrize("n", [2, 7, 32, 64, 100, 128, 256, 300, 384, 512, 1000, 1024, 2048, 4096])
@pytest.mark.parametrize("prec", [B.BFM_FP32, B.BFM_FP64])
def test_candidates_are_valid_shapes(n, prec):
    for kind in KINDS:
        cand = B.bfm_tune_candidates(kind, n, prec)
        if kind in ROW_KINDS and n <= 256:
            assert cand == []                  # short lines never take the row kernel
            continue
        assert len(set(cand)) == len(cand)
        assert B.bfm_tune_default(kind, n, prec) in cand
        for K, W in cand:
            assert K <= n and K in ((16, 32) if kind in ROW_KINDS else (1, 2, 4, 8, 12, 16, 24, 32))
            G = _next_pow2(-(-n // K))
            assert G <= 512
            if kind in ROW_KINDS:
                assert G >= 32                 # row groups are whole warps
            if W:
                assert W * G <= 512 and W * G >= 32
                if kind in (B.CT_KIND_TILE_COLS, B.CT_KIND_ROW_COLS):
                    assert W & (W - 1) == 0    # interleaved tiles: a power of two
                if G < 32:
                    assert (W * G) % 32 == 0


def test_set_get_clear():
    n = 128
    K0, W0 = B.bfm_tune_default(B.CT_KIND_TILE_COLS, n)
    assert B.bfm_tune_get(B.CT_KIND_TILE_COLS, n) == (K0, W0, False)
    other = [c for c in B.bfm_tune_candidates(B.CT_KIND_TILE_COLS, n) if c != (K0, W0)][0]
    B.bfm_tune_set(B.CT_KIND_TILE_COLS, n, *other)
    assert B.bfm_tune_get(B.CT_KIND_TILE_COLS, n) == (other[0], other[1], True)
    # other kinds, lengths and precisions keep their defaults
    assert B.bfm_tune_get(B.CT_KIND_TILE_ROWS, n)[2] is False
    assert B.bfm_tune_get(B.CT_KIND_TILE_COLS, n, B.BFM_FP64)[2] is False
    B.bfm_tune_clear()
    assert B.bfm_tune_get(B.CT_KIND_TILE_COLS, n) == (K0, W0, False)


def test_set_rejects_non_candidates():
    for bad in ((3, 0), (16, 3), (24, 0), (64, 0)):
        with pytest.raises(B.BfmError) as e:
            B.bfm_tune_set(B.CT_KIND_TILE_COLS, 128, *bad)
        assert e.value.status == B.BFM_ERR_INVALID_ARG
    with pytest.raises(B.BfmError):
        B.bfm_tune_set(B.CT_KIND_ROW, 128, 16, 0)          # 128-cell rows take tiles


def test_pick_keeps_default_within_margin():
    assert B.bfm_tune_pick([1.0, 0.99, 1.2], 0) == 0        # 1% faster: noise
    assert B.bfm_tune_pick([1.0, 0.97, 1.2], 0) == 1        # 3% faster
    assert B.bfm_tune_pick([1.0, 0.97, 0.5], 0) == 2        # the fastest wins
    assert B.bfm_tune_pick([-1.0, 0.97, 0.98], 0) == 1      # default not measured
    assert B.bfm_tune_pick([1.0, 0.9], -1) == 1             # no default among them
    assert B.bfm_tune_pick([1.0, 0.9], 0, margin=0.2) == 0
    assert B.bfm_tune_pick([-1.0, -1.0], 1) == 1            # nothing measured: default


def test_passes_of_a_solve():
    R, C, T = B.CT_KIND_ROW, B.CT_KIND_TILE_COLS, B.CT_KIND_TILE_ROWS
    RC = B.CT_KIND_ROW_COLS
    assert B.bfm_tune_passes((4096, 4096)) == [(R, 4096)]   # long columns: rows of a transposed copy
    # columns of more than 256 cells: the row kernel on interleaved tiles
    assert B.bfm_tune_passes((512, 512)) == [(R, 512), (RC, 512)]
    assert B.bfm_tune_passes((64, 128)) == [(T, 128), (C, 64)]
    assert B.bfm_tune_passes((384, 384, 384)) == [(R, 384), (RC, 384)]
    assert B.bfm_tune_passes((300, 5, 3)) == [(T, 3), (C, 5), (RC, 300)]
    # row-kernel tiles of 1024-cell columns would hold fewer than 32 bytes per
    # position: the tile kernel, or (FP64) rows of a transposed copy
    assert B.bfm_tune_passes((1024, 3)) == [(T, 3), (C, 1024)]
    assert B.bfm_tune_passes((1024, 3), B.BFM_FP64) == [(T, 3), (R, 1024)]
    assert B.bfm_tune_passes((2048, 512)) == [(R, 512), (R, 2048)]
    assert B.bfm_tune_passes((2048, 512), batched=True) == [(R, 512), (C, 2048)]
