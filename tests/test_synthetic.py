"""The seeded input generators: Philox known-answer vectors, SU(3) links, Gaussian statistics."""
import numpy as np

import synthetic


def test_philox_known_answer_vectors():
    # Philox4x32-10 test vectors published with the Random123 library (Salmon et al., SC11)
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
        ((0xffffffff,) * 4, (0xffffffff, 0xffffffff), (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
        ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
         (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
    ]
    for ctr, key, expect in cases:
        out = synthetic.philox4x32_10(*ctr, *key)
        assert tuple(int(v) for v in out) == expect


def test_philox_fields_are_su3_and_gaussian():
    U = synthetic.gauge_field_philox((4, 4, 4, 4), 0.4, 3)
    assert np.abs(np.conj(np.swapaxes(U, -1, -2)) @ U - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    e = synthetic.gaussian_source_philox((8, 8, 8, 8), 4)
    for part in (e.real, e.imag):
        assert abs(part.mean()) < 0.02 and abs(part.std() - 1) < 0.02
    # different seeds and streams give different fields
    assert np.abs(synthetic.gaussian_source_philox((2, 2, 2, 2), 5) - synthetic.gaussian_source_philox((2, 2, 2, 2), 6)).min() > 0


def test_philox_gauge_chunking_is_invisible():
    a = synthetic.gauge_field_philox((4, 2, 2, 4), 0.3, 11, chunk=7)
    b = synthetic.gauge_field_philox((4, 2, 2, 4), 0.3, 11)
    assert np.array_equal(a, b)
