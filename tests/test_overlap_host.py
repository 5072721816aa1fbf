"""Host logic of the overlap building blocks (no GPU): the library's Chebyshev
coefficients of the sign approximation (Sec. 2.3) equal the oracle's,
computed independently from the same definition, term count included."""
import numpy as np
import pytest

from helpers import ensure_library


@pytest.mark.parametrize("eps,delta", [(0.2, 1e-5), (0.05, 1e-5), (0.02, 1e-7)])
def test_sign_coefficients_match_oracle(orc, eps, delta):
    ensure_library()
    from paper_2201_09004_b300 import lib
    c, dev = lib.chebyshev_sign(eps, delta)
    co, devo = orc.chebyshev_sign_coeffs(eps, delta)
    assert len(c) == len(co)
    assert np.max(np.abs(np.array(c) - co)) < 1e-12
    assert dev <= delta and abs(dev - devo) < 1e-12


def test_sign_coefficients_reject_bad_arguments():
    ensure_library()
    from paper_2201_09004_b300 import lib
    for eps, delta in [(0.0, 1e-5), (1.0, 1e-5), (0.1, 0.0)]:
        with pytest.raises(lib.LqError) as e:
            lib.chebyshev_sign(eps, delta)
        assert e.value.code == lib.LQ_EINVAL
    with pytest.raises(lib.LqError):
        lib.chebyshev_sign(0.001, 1e-12, max_order=64)
