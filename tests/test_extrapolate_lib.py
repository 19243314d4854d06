"""The library's energy extrapolation (host code behind the C-ABI, no GPU needed) against
the oracle's fits on seeded data: exact power laws, noisy ones, and the rejected cases."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def P():
    from paper_1507_00161_gb300.build import build
    build()
    import paper_1507_00161_gb300 as P
    return P


def _sets():
    rng = np.random.default_rng(11)
    out = []
    for k in range(12):
        n = int(rng.integers(4, 12))
        M = np.sort(rng.choice(np.arange(64, 8193), size=n, replace=False)).astype(float)
        e_inf = rng.uniform(-320.0, -20.0)
        x2 = -rng.uniform(0.2, 2.5)
        x1 = rng.uniform(0.5, 50.0) * 1024.0 ** (-x2) * 1e-2
        noise = 0.0 if k % 3 == 0 else 10.0 ** rng.uniform(-6, -3)
        E = e_inf + x1 * M ** x2 + noise * rng.standard_normal(n)
        out.append((M, E))
    return out


@pytest.mark.parametrize("i", range(12))
def test_power_fit_matches_oracle(P, i):
    from oracle.extrapolate import fit_power
    M, E = _sets()[i]
    try:
        ref = fit_power(M, E)
    except ValueError:
        with pytest.raises(P.DmrgError) as e:
            P.extrapolate(M, E, P.FIT_POWER)
        assert e.value.code == P.DMRG_ENOCONV
        return
    got = P.extrapolate(M, E, P.FIT_POWER)
    scale = np.max(np.abs(E))
    # the same least-squares minimum: residuals agree to rounding, parameters to the
    # flatness of the minimum in the exponent
    assert abs(got[3] - ref[3]) <= 1e-6 * ref[3] + 1e-9 * scale
    assert abs(got[0] - ref[0]) <= 1e-6 * scale
    assert abs(got[2] - ref[2]) <= 1e-5 * abs(ref[2])
    fit_g = got[0] + got[1] * M ** got[2]
    fit_r = ref[0] + ref[1] * M ** ref[2]
    assert np.max(np.abs(fit_g - fit_r)) <= 1e-6 * scale


@pytest.mark.parametrize("i", range(12))
def test_quadratic_fit_matches_oracle(P, i):
    from oracle.extrapolate import fit_quadratic
    M, E = _sets()[i]
    ref = fit_quadratic(M, E)
    got = P.extrapolate(M, E, P.FIT_QUADRATIC)
    scale = np.max(np.abs(E))
    assert abs(got[0] - ref[0]) <= 1e-10 * scale
    x = 1.0 / M
    fit_g = got[0] + got[1] * x + got[2] * x * x
    fit_r = ref[0] + ref[1] * x + ref[2] * x * x
    assert np.max(np.abs(fit_g - fit_r)) <= 1e-10 * scale
    assert abs(got[3] - ref[3]) <= 1e-8 * max(ref[3], 1e-6 * scale)


def test_rejected_inputs_match_oracle(P):
    from oracle.extrapolate import fit_power
    bad = [(np.array([256.0, 512.0]), np.array([1.0, 2.0])),
           (np.array([256.0, 256.0, 512.0]), np.array([1.0, 2.0, 3.0])),
           (np.array([256.0, 0.0, 512.0]), np.array([1.0, 2.0, 3.0])),
           (np.array([256.0, 384.0, 512.0]), np.array([1.0, np.nan, 3.0]))]
    for M, E in bad:
        with pytest.raises(ValueError):
            fit_power(M, E)
        for kind in (P.FIT_POWER, P.FIT_QUADRATIC):
            with pytest.raises(P.DmrgError) as e:
                P.extrapolate(M, E, kind)
            assert e.value.code == P.DMRG_EINVAL
    with pytest.raises(P.DmrgError) as e:
        P.extrapolate(np.array([1.0, 2.0, 3.0]), np.zeros(3), 7)
    assert e.value.code == P.DMRG_EINVAL
    M = np.array([256.0, 512.0, 1024.0, 2048.0])
    with pytest.raises(ValueError):
        fit_power(M, -1e-3 * M)
    with pytest.raises(P.DmrgError) as e:
        P.extrapolate(M, -1e-3 * M, P.FIT_POWER)
    assert e.value.code == P.DMRG_ENOCONV
