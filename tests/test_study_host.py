"""Host logic of the LUT-length study driver: the prime table lengths it sweeps."""

from paper_2004_04049_gb300 import study


def test_is_prime_against_trial_division():
    def slow(n):
        return n >= 2 and all(n % d for d in range(2, int(n ** 0.5) + 1))
    assert [n for n in range(2000) if study.is_prime(n)] == [n for n in range(2000) if slow(n)]
    assert study.is_prime(10007) and not study.is_prime(10007 * 10009)
    assert study.next_prime(10000) == 10007


def test_prime_grid():
    g = study.prime_grid(64, 24, points=12)
    assert all(study.is_prime(L) for L in g)
    assert 10007 in g and g == sorted(set(g)) and g[0] == 2 and g[-1] >= 4 * 24 * 64 * 64
    assert study.next_prime(24) in g and study.next_prime(64) in g
