"""The counter-based radiance generator that both sides of the full-size
coverage test draw from: SplitMix64's published first outputs, and the numpy
and torch versions agreeing bit for bit."""
import numpy as np

from paper_2605_24290_gb300 import synthetic as S


def test_splitmix64_known_outputs():
    # the first three outputs of SplitMix64 seeded with 0 (Steele, Lea and
    # Flood 2014; the generator Java's SplittableRandom and Vigna publish)
    with np.errstate(over="ignore"):
        z = S._splitmix64_np(np.array([1, 2, 3], np.uint64))
    assert [int(x) for x in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_hashed_radiance_numpy_equals_torch():
    import torch
    K = 777
    rows = [0, 3, 12, 39]
    a = S.hashed_radiance_rows(rows, K)
    b = S.hashed_radiance_torch(torch, 40, K, "cpu", rows_per_pass=7)
    assert a.dtype == np.float32 and b.dtype == torch.float32
    np.testing.assert_array_equal(a, b[rows].numpy())
    assert a.min() >= -1.0 and a.max() < 1.0
    assert abs(float(a.mean())) < 0.05


def test_film_frequencies_start_at_powers_of_two():
    """The receiver encoding's frequencies start at 2^f along each axis
    (App. E.4), F bands per axis."""
    import numpy as np
    from paper_2605_24290_gb300 import synthetic as S
    w = S.film_frequencies(6)
    assert w.shape == (18, 3) and w.dtype == np.float32
    for d in range(3):
        for f in range(6):
            row = np.zeros(3, np.float32)
            row[d] = 2.0 ** f
            np.testing.assert_array_equal(w[d * 6 + f], row)
