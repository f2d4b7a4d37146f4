"""The kernels' Table 1 start-index routine (Section 3), evaluated on the host
through the C ABI, against the paper's worked example and the plain
definition (smallest class-r multiple of P that is >= max(M, P^2))."""
import numpy as np
import pytest

import oracle
import oracle_checks as C
from paper_2310_17746_gb300 import binding


def test_worked_example():
    ex = C.golden("table1_worked_example.json")
    # the chunk's index 0 is the group base value; M is the chunk start value
    B = ex["group_base_value"]
    id1, id5 = binding.table1_start(B, ex["M"], ex["P"])
    assert (id1, id5) == (ex["id_1"], ex["id_5"])
    assert B + 6 * id1 + 1 == ex["start_value_1"]
    assert B + 6 * id5 + 5 == ex["start_value_5"]


def _check(B, M, P):
    id1, id5 = binding.table1_start(B, M, P)
    assert B + 6 * id1 + 1 == oracle.first_class_multiple(M, P, 1, True), (B, M, P)
    assert B + 6 * id5 + 5 == oracle.first_class_multiple(M, P, 5, True), (B, M, P)


def test_all_twelve_cells_small():
    """Every (P mod 6, Q mod 6) cell of Table 1, many times over."""
    primes = [p for p in range(5, 2000) if C.td_is_prime(p)]
    rng = np.random.default_rng(1)
    cells = set()
    for P in primes:
        for _ in range(12):
            B = 6 * int(rng.integers(0, 10**6))
            M = B + int(rng.integers(0, 6 * 4096))
            _check(B, M, P)
            Mp = max(M, P * P)
            cells.add((P % 6, ((Mp - 1) // P * P) % 6))
    assert len(cells) == 12


@pytest.mark.parametrize("scale", [10**12, 10**15, 10**18, 2**62])
def test_large_values(scale):
    rng = np.random.default_rng(scale % 1000)
    big_primes = [4294967291, 3037000493, 2147483647, 1000000007, 999999937, 65521, 23, 29]
    for P in big_primes:
        for _ in range(40):
            B = 6 * (int(rng.integers(0, scale // 6)))
            M = B + int(rng.integers(0, 6 * (1 << 20)))
            if M >= 2**63 or max(M, P * P) - B >= 2**62:
                continue
            _check(B, M, P)


def test_tile_path_m_equals_b():
    """M == B is the kernels' per-tile case (32-bit path once P^2 <= B)."""
    rng = np.random.default_rng(9)
    primes = [p for p in range(5, 3000) if C.td_is_prime(p)] + [65521, 999983, 2147483647, 3037000493]
    for P in primes:
        for _ in range(10):
            B = 6 * int(rng.integers(0, 10**17 // 6))
            if max(B, P * P) - B < 2**62:
                _check(B, B, P)
        if P * P < 2**62:  # the entry's argument bound: max(M, P^2) - B < 2^62
            _check(0, 0, P)
        B = 6 * ((P * P) // 6)  # tile base just below P^2
        _check(B, B, P)
        _check(B + 6, B + 6, P)


def test_square_start():
    """Section 2.4: a prime's strikes start at its square (5 -> 25 / 35, 7 -> 49 / 77)."""
    for P, s1, s5 in ((5, 25, 35), (7, 49, 77), (11, 121, 143), (13, 169, 221)):
        id1, id5 = binding.table1_start(0, 0, P)
        assert 6 * id1 + 1 == s1 and 6 * id5 + 5 == s5


def test_invalid_arguments():
    for args in ((1, 1, 7), (0, 0, 4), (0, 0, 9), (12, 6, 7), (0, 0, 3)):
        with pytest.raises(binding.SieveError):
            binding.table1_start(*args)


def _check_inverse(B, P):
    id1, id5 = binding.inverse6_start(B, P)
    assert B + 6 * id1 + 1 == oracle.first_class_multiple(B, P, 1, True), (B, P)
    assert B + 6 * id5 + 5 == oracle.first_class_multiple(B, P, 5, True), (B, P)
    assert (id1, id5) == binding.table1_start(B, B, P), (B, P)


def test_inverse6_start_matches_definition_and_table1():
    """The one-lane band's starts from (-r / 6) mod P equal the smallest
    class-r multiple >= B (and Table 1's tile starts) whenever P^2 <= B, in
    every residue of B / 6 mod P and P mod 6."""
    rng = np.random.default_rng(17)
    primes = [p for p in range(5, 3000) if C.td_is_prime(p)]
    seen = set()
    for P in primes:
        for _ in range(8):
            B = 6 * int(rng.integers((P * P + 5) // 6, 10**15))
            _check_inverse(B, P)
            seen.add((P % 6, (B // 6) % P == 0))
        B = 6 * ((P * P + 5) // 6)  # the first tile base at or above P^2
        _check_inverse(B, P)
        _check_inverse(6 * P * P, P)  # B / 6 = 0 (mod P)
    assert seen >= {(1, False), (5, False)}
    for P in (65521, 999983, 1000003, 2147483647, 2147483629):
        for scale in (10**13, 10**18, 2**62):
            low = -(-P * P // 6)  # B >= P^2
            if low >= scale // 6:
                continue
            for _ in range(20):
                _check_inverse(6 * int(rng.integers(low, scale // 6)), P)


def test_inverse6_start_rejects_outside_its_domain():
    for B, P in ((6, 7), (48, 7), (100 * 6 + 1, 7), (6 * 10**6, 4), (6 * 10**6, 9), (2**62, 2**31 + 11)):
        with pytest.raises(binding.SieveError):
            binding.inverse6_start(B, P)
