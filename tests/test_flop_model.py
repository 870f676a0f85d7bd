"""The benchmark's FLOP model rests on counted operations, not typed-in constants.

bench.py composes the algorithmic FLOPs of a solve from the operation counts
of its linear-algebra primitives (14 x 14 block products, block-tridiagonal
rows, 7 x 7 Cholesky solves).  Here the FP64 oracle runs those primitives on
its FLOP-counting scalar (Sec. II-B / III-B's PCG and Eq. 5-6 blocks are built
from them) and the counts must equal the numbers bench.py uses.
"""
import bench
from paper_2510_07625_gb300 import inputs as I


def test_primitive_counts_match_the_oracle_counter(oracle):
    got = oracle.count_flops(I.arm7())
    assert bench.FLOP_PRIM["block_product_14"] == got["block_product_14"] == 2 * 14 ** 3
    assert bench.FLOP_PRIM["blocktri_row_14"] == got["blocktri_row_14"]
    assert bench.FLOP_PRIM["cholesky_solve_7"] == got["cholesky_solve"]


def test_pcg_row_composition():
    # one middle block row of S u is three block-vector products
    assert 3 * bench.BLOCK_MV_14 == 1176
    # the factored stair costs two diagonal-block products plus the off-diagonal
    # part of a row; with S u and the vector updates about 2.6 kFLOP a row
    assert 2400 < bench.PCG_ROW < 2800


def test_counter_counts_multiply_adds_as_two(oracle):
    # a 14 x 14 product is 14^3 multiply-adds; the tangent pass of an RNEA
    # costs more than the value pass it rides on
    got = oracle.count_flops(I.arm7())
    assert got["rnea_tangent_and_value"] > 2 * got["rnea"]
    assert got["fk_and_tangent"] > 2 * got["fk"]
