"""model_shots_static: forward modelling for callers that cannot allocate
device memory (its temporaries live in the library's static device array).

It must give the records model_shots gives, on two calls in a row (the
array keeps the previous call's contents, so the second call checks that the
state is cleared), and reject problems larger than the array.  This file is
collected last so a run that stops at the first failure has already run every
other test.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import f32, f32_geom, gpu_ctx, rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["config1", "ragged"])
def test_static_matches_model_shots_twice(name, monkeypatch):
    c = synth.config1_case() if name == "config1" else synth.tiny_case(nz=37, nx=141, nt=150, nb=20,
                                                                      n_shots=3, seed=8)
    ctx = gpu_ctx(c)
    from paper_2403_17518_gb300.ops import model_shots_static

    v, geom = to_dev(f32(c.v_true)), f32_geom(c.geom)
    ref = to_host(ctx.model_shots(v, geom))
    # model_shots pinned to the kernel the static call runs (one step per
    # launch, cp.async variant 1), in a fresh context (the variant choice is
    # made once per context and geometry): the same bits.
    monkeypatch.setenv("DHFWI_TIME_BLOCK", "0")
    monkeypatch.setenv("DHFWI_STEP_VARIANT", "1")
    ctx1 = gpu_ctx(c)
    ref1 = to_host(ctx1.model_shots(v, geom))
    ctx1.close()
    monkeypatch.delenv("DHFWI_TIME_BLOCK")
    monkeypatch.delenv("DHFWI_STEP_VARIANT")
    for _ in range(2):
        d = to_host(model_shots_static(c.nz, c.nx, c.h, c.dt, c.nb, v, geom))
        assert rel_l2(d, ref) <= 1e-5
        assert np.array_equal(d, ref1)
    # A different model in between, then the first again: nothing carries over.
    model_shots_static(c.nz, c.nx, c.h, c.dt, c.nb, to_dev(f32(c.v_init)), geom)
    d = to_host(model_shots_static(c.nz, c.nx, c.h, c.dt, c.nb, v, geom))
    assert rel_l2(d, ref) <= 1e-5
    assert np.array_equal(d, ref1)


def test_static_rejects_problems_beyond_the_array():
    c = synth.config2_case(n_shots=32, nt_range=(100, 120))
    gpu_ctx(synth.tiny_case())
    from paper_2403_17518_gb300.ops import DhfwiError, model_shots_static

    with pytest.raises(DhfwiError, match="ARG.*static array"):
        model_shots_static(c.nz, c.nx, c.h, c.dt, c.nb, to_dev(c.v_true), c.geom)
