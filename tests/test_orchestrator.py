"""The RGF / DDRGF choice for n_domains = 0 (negf_auto_domains: host
arithmetic only, so it runs without a GPU)."""
import pytest


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_2605_19910_gb300 as P
    return P


def test_many_energies_choose_plain_rgf(P):
    # the benchmark workload fills the GPU with energies alone
    assert P.negf_auto_domains([64] * 64, 3, 512, 152) == 1
    assert P.negf_auto_domains([48] * 128, 3, 256, 152) == 1
    assert P.negf_auto_domains([32] * 256, 5, 1024, 152) == 1


def test_few_energies_long_chain_choose_ddrgf(P):
    d1 = P.negf_auto_domains([64] * 1024, 3, 1, 152)
    d2 = P.negf_auto_domains([64] * 4096, 3, 1, 152)
    assert d1 > 1 and d2 >= d1
    for d in (d1, d2):
        assert d & (d - 1) == 0                      # a power of two


def test_pairs_keep_at_least_four_w_layers(P):
    for N in range(2, 64):
        for band_n in (3, 5):
            w = (band_n - 1) // 2
            d = P.negf_auto_domains([16] * N, band_n, 1, 152)
            assert d == 1 or N // d >= 4 * w, (N, band_n, d)


def test_more_energies_never_increase_the_domain_count(P):
    prev = None
    for nE in (1, 2, 8, 64, 256, 1024, 4096):
        d = P.negf_auto_domains([96] * 512, 3, nE, 152)
        if prev is not None:
            assert d <= prev, (nE, d, prev)
        prev = d
    assert prev == 1


def test_invalid_arguments_fall_back_to_rgf(P):
    assert P.negf_auto_domains([], 3, 1, 152) == 1
    assert P.negf_auto_domains([8, 8], 3, 0, 152) == 1
    assert P.negf_auto_domains([8, 8], 3, 1, 0) == 1


def test_paper_cost_model_choices():
    """negf_ddrgf_model (Eq. cost_model_DDRGF with Eq. cost_model_RGF, GPU
    wave factors): plain RGF when the energies fill the GPU, recursive DDRGF
    with valid levels for few energies on long chains."""
    import paper_2605_19910_gb300 as P
    # 512 energies of 64 x 64 fill the GPU: plain RGF
    nd, lv, crgf, cdd = P.negf_ddrgf_model([64] * 64, 3, 512, 152, 3.0)
    assert nd == 1 and lv == [] and cdd == crgf
    # one energy on a long chain: DDRGF, deeper levels that each cut the
    # previous level's separators into pairs of at least two nodes
    for N, b, w in [(1024, 64, 1), (4096, 32, 1), (256, 32, 2)]:
        nd, lv, crgf, cdd = P.negf_ddrgf_model([b] * N, 2 * w + 1, 1, 152, 3.0)
        assert 1 < nd <= 128 and N // nd >= 3 * w
        assert cdd < crgf
        prev = nd
        for pairs in lv:
            assert 1 <= pairs and 2 * pairs <= prev
            prev = pairs
    # the model's RGF cost is Eq. cost_model_RGF with r_LU = r_inv, r_GETRS = 1
    _, _, crgf, _ = P.negf_ddrgf_model([64] * 100, 3, 1, 152, 2.5)
    assert abs(crgf - (100 * (4 + 2.5 + 3) - (4 + 2))) < 1e-9
    # more energies leave less room for concurrent tasks: no more pairs than with fewer
    n1 = P.negf_ddrgf_model([64] * 1024, 3, 1, 152, 3.0)[0]
    n64 = P.negf_ddrgf_model([64] * 1024, 3, 64, 152, 3.0)[0]
    n512 = P.negf_ddrgf_model([64] * 1024, 3, 512, 152, 3.0)[0]
    assert n1 >= n64 >= n512
