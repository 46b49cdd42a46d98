"""The uneven batch recipe (synthetic.batch_specs) is seeded and stays in range."""
from synthetic import batch_specs


def test_batch_recipe_is_seeded_and_in_range():
    a, b = batch_specs(16, seed=0), batch_specs(16, seed=0)
    assert a == b and len(a) == 16
    assert batch_specs(16, seed=1) != a
    for i, sp in enumerate(a):
        assert 64 <= sp.N1 <= 256 and 64 <= sp.N2 <= 256
        assert sp.N3 in (31, 64, 128, 191) and sp.k in (3, 5)
        assert sp.sigma in (0.05, 0.1) and sp.p_t in (0.0, 0.05, 0.10) and sp.p_s == 0.05
        assert sp.regions == max(4, sp.N1 * sp.N2 // 2048) and sp.endmembers == 5 and sp.seed == 1000 + i
