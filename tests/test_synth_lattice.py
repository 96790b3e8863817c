"""The committed Korobov generators equal what the P_2 search finds (the
table only saves the search time of the large reference rule)."""
from paper_2005_06848_gb300 import synth


def test_korobov_table_matches_the_search():
    for (n, dim), a in synth.KOROBOV_TABLE.items():
        assert synth.korobov_search(n, dim) == a, (n, dim)


def test_generator_is_coprime_and_cached():
    a = synth.korobov_generator(1024, 3)
    import math
    assert math.gcd(a, 1024) == 1
    assert synth.korobov_generator(1024, 3) == a
