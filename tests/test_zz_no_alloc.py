"""lbve_fields_host_fixed: the host copy of the fields that allocates no device memory.

Callers that cannot allocate device memory after their set-up (a fixed device-memory budget, an
application whose own pool owns the GPU, a stepping loop that must not pay an allocation's device-wide
synchronisation) use this entry point instead of lbve_fields, which allocates its staging buffer on first
use.  It stages through one fixed device array inside the library.  This file sorts last so that a run
stopping at the first failure has already run every other test; it needs nothing from them.
"""
import numpy as np
import pytest

from paper_1504_06123_gb300 import lbve as L

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALL = L.LBVE_FIELD_RHO | L.LBVE_FIELD_U | L.LBVE_FIELD_SIGMA | L.LBVE_FIELD_KAPPA | L.LBVE_FIELD_N1
TOL = 1e-5   # the parity tolerance of the plain FP32 form; the two copies are expected to be identical


def _check_same(fixed, ref):
    assert fixed.shape == ref.shape
    np.testing.assert_allclose(fixed, ref, rtol=TOL, atol=0)
    assert np.array_equal(fixed, ref)


def test_fixed_staging_matches_lbve_fields_on_consecutive_calls():
    ch = L.Channel(L.make_desc(L.LBVE_D2Q9, 7, 19, G_inf=0.01, tau=40.0, gamma_c=0.1, g=(1e-5, 0, 0), C=8, B=3,
                               precision=L.LBVE_F64, hist_storage=L.LBVE_F32))
    ch.step(25)
    first = L.lbve_fields_host_fixed(ch.h, ALL)
    _check_same(first, L.lbve_fields(ch.h, ALL))
    # second call right after the first, with a different field selection (smaller and offset): the array
    # keeps the previous call's contents, which must not leak into this result
    second = L.lbve_fields_host_fixed(ch.h, L.LBVE_FIELD_SIGMA | L.LBVE_FIELD_N1)
    _check_same(second, L.lbve_fields(ch.h, L.LBVE_FIELD_SIGMA | L.LBVE_FIELD_N1))
    # and once more after the flow has moved on
    ch.step(10)
    third = L.lbve_fields_host_fixed(ch.h, ALL)
    _check_same(third, L.lbve_fields(ch.h, ALL))
    assert not np.array_equal(third, first)
    ch.close()


def test_fixed_staging_rejects_requests_beyond_its_size():
    # 1024 x 512 nodes: all fields are 11 x 524288 doubles, more than the fixed array's 2^21
    ch = L.Channel(L.make_desc(L.LBVE_D2Q9, 1024, 512, C=4, B=1, precision=L.LBVE_F64, hist_storage=L.LBVE_F32))
    assert L.lbve_fields_count(ch.h, ALL) > L.LBVE_FIXED_STAGING_DOUBLES
    with pytest.raises(L.LbveError) as e:
        L.lbve_fields_host_fixed(ch.h, ALL)
    assert e.value.status == L.LBVE_ETOOBIG
    # a selection that fits still works
    u = L.lbve_fields_host_fixed(ch.h, L.LBVE_FIELD_U)
    _check_same(u, L.lbve_fields(ch.h, L.LBVE_FIELD_U))
    ch.close()
