"""The per-kernel profiler of the C-ABI (negf_profile_read and
negf_profile_read_issued): the method's flop counts of one solve, and the
flops the units execute, whose ratio is fixed by each product kernel's form
(three real products per complex one in the FP64 3M product; L (L + 1) / 2
BF16 slice products per useful one in the exact-slice product with L
slices, on shapes that fill its tiles)."""
import pytest

from gpu_parity import to_dev
from workloads import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_2605_19910_gb300 as P
    return P


@pytest.mark.parametrize("precision,bits,ratio", [("fp64", 0, 0.75), ("mixed", 35, 15.0), ("mixed", 48, 28.0)])
def test_profile_counts_of_one_solve(P, precision, bits, ratio):
    import torch
    N, b, nE = 5, 64, 8
    prob = make_problem(N, b=b, w=1, n_energies=nE, eta=1e-3, seed=17)
    Hp, sL, sR, E = to_dev(prob, torch)
    plan = P.Plan(prob.sizes, 3, nE, precision=precision, product_bits=bits)
    assert P.negf_profile_enable(plan.handle, 1) == P.NEGF_OK
    plan.solve(Hp, sL, sR, E)
    first = P.negf_profile_read_issued(plan.handle)
    plan.solve(Hp, sL, sR, E)
    second = P.negf_profile_read(plan.handle)
    P.negf_profile_enable(plan.handle, 0)
    plan.close()

    inv = first["zinv_gj_kernel"]
    assert inv[3] >= N and inv[0] > 0
    assert inv[1] == pytest.approx(N * nE * 8.0 * b ** 3)     # one b x b inverse per layer and energy
    assert inv[2] == pytest.approx(inv[1])
    prod = first["zgemm_tc_kernel" if precision == "mixed" else "zgemm_f64_kernel"]
    other = first["zgemm_f64_kernel" if precision == "mixed" else "zgemm_tc_kernel"]
    assert prod[3] > 0 and prod[0] > 0
    assert other[1] == 0 and other[2] == 0   # at most empty products (lead terms) on the other kernel
    assert prod[1] > 0 and prod[1] % (8.0 * b ** 3 * nE) == 0   # whole 64 x 64 x 64 products
    assert prod[2] == pytest.approx(ratio * prod[1])
    # the plain read reports the same counts for the same call
    for k, v in second.items():
        assert v[1] == pytest.approx(first[k][1]) and v[2] == first[k][3]
