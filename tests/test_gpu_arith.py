"""The kernels' FP64 products, quotients and square roots computed on the
integer pipes (correctly rounded from 64-bit integer arithmetic on the
significands, with the FP64 instruction for operands or results outside the
normal range) against the FP64 hardware operations, bit for bit, on 3 x 2^24
hashed operand pairs each: any bit pattern, random values over 81 binades,
and significands with trailing zeros (exact results and ties)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1206_5878_gb300 as lib
    lib.load()
    return lib


@pytest.mark.parametrize("op", [0, 1, 2], ids=["mul", "div", "sqrt"])
def test_integer_pipe_fp64_equals_hardware(g, op):
    assert g.check_arith(op, 3 << 24, seed=12345 + op) == 0


def test_check_arith_argument_checks(g):
    with pytest.raises(g.CMCError):
        g.check_arith(3, 10)
