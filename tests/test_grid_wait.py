"""The bounded grid-wide wait of the persistent sweep kernels, on the GPU.

A two-CTA cooperative kernel meets at one phase boundary.  When one CTA never
arrives (a flag that nothing sets), the other must give up after the wait
limit, report it through the error word, and leave the context usable.
"""
import time

import numpy as np
import pytest

from synth import hubbard_chain

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2604_16118_gb300 import build, native
    build.build()
    return native


@pytest.fixture(scope="module")
def ctx(nat):
    return nat.Context(0)


def test_all_arrive_no_timeout(nat, ctx):
    assert nat.check_grid_wait(ctx, -1) is False


@pytest.mark.parametrize("skip", [0, 1])
def test_missing_cta_times_out_and_context_survives(nat, ctx, skip):
    t0 = time.perf_counter()
    assert nat.check_grid_wait(ctx, skip) is True
    dt = time.perf_counter() - t0
    assert 0.5 < dt < 30.0
    # the context still runs the solver's kernels correctly afterwards
    wl = hubbard_chain(L=3, n_up=1, n_dn=1, U=4.0)
    x = nat.mps_create(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn)
    n2 = nat.dot(ctx, x, x)
    assert np.isclose(n2, 1.0, rtol=1e-14)
    assert nat.check_grid_wait(ctx, -1) is False


def test_rejects_bad_cta_index(nat, ctx):
    with pytest.raises(nat.BsmpsError):
        nat.check_grid_wait(ctx, 2)
