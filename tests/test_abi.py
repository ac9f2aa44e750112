"""The C ABI: the library builds, loads, exports every declared symbol, and
its host-side setup (KL builder, midpoint transfer) agrees with the oracle
through invariants (no GPU needed)."""
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mlq():
    from paper_2105_02007_gb300 import build

    build.build()
    from paper_2105_02007_gb300 import mlq as m

    return m


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mlq.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(mlq_\w+)\s*\(", src, flags=re.M)))


def test_header_symbols_exported(mlq):
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(mlq._lib, s), s
    assert set(syms) == set(mlq.EXPORTED)


def test_error_strings_and_bad_arguments(mlq):
    assert mlq._lib.mlq_strerror(0) == b"ok"
    assert mlq._lib.mlq_strerror(-1) == b"invalid argument"
    with pytest.raises(mlq.MLQError):
        mlq.build_kl(1, 0.09, 0.04, 4)          # m < 2
    with pytest.raises(mlq.MLQError):
        mlq.build_kl(5, 0.09, 0.04, 26)         # K > n


def test_product_kl_matches_oracle_invariants(mlq):
    m, K = 17, 10
    pm, pl = mlq.build_kl(m, 0.09, 0.04, K)
    mesh = O.mesh2d(m)
    om, ol = O.kl_build(mesh, 0.09, 0.04, K)
    assert np.allclose(pl, ol, rtol=1e-11, atol=1e-15)
    rp, ci, mv, _ = O.assemble(mesh)
    M = O.csr_to_dense(rp, ci, mv, mesh.n)
    assert np.allclose(pm.T @ M @ pm, np.diag(pl), atol=1e-13)
    # the covariance the modes represent is basis independent
    assert np.allclose(pm @ pm.T, om @ om.T, atol=1e-12)


def test_product_centroid_table_matches_oracle(mlq):
    fine = O.mesh2d(33)
    modes, _ = O.kl_build(fine, 0.09, 0.04, 5)
    for mc in (33, 17, 9, 3):
        coarse = O.mesh2d(mc)
        ref = O.centroid_table(fine, modes, coarse)
        got = mlq.centroid_table(33, modes, mc)
        assert np.allclose(got, ref, rtol=0, atol=1e-15)
