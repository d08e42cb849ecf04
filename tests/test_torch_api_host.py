"""Host logic of the autograd layer without a GPU: the parameter vector follows the plan's
gradient layout, and uploading a vector rebuilds every transform with its structure (n, core,
kind, layer parities, K) unchanged and the new values in place."""

import numpy as np

import synth
from paper_2505_23618_gb300 import torch_api as T


class FakePlan:
    """Stands in for a Plan: its transform table and gradient layout (angles per band, K*K per
    post block, n*n per dense transform, nothing for a plain core)."""

    def __init__(self, tfs):
        self.tfs = list(tfs)
        sizes = []
        for t in self.tfs:
            if t.kind == synth.KIND_BAND:
                sizes.append(len(t.angles))
            elif t.kind in (synth.KIND_POST, synth.KIND_DENSE):
                sizes.append(t.q.size)
            else:
                sizes.append(0)
        self._param_layout = [0] + list(np.cumsum(sizes))
        self.uploads = []

    def update_params(self, tfs):
        self.uploads.append(tfs)
        self.tfs = list(tfs)


def table():
    rng = np.random.default_rng(5)
    return [synth.random_band(rng, 16, synth.CORE_DST3, [0, 1, 0]),
            synth.Tf(n=8, core=synth.CORE_DCT2),
            synth.random_post(rng, 32, synth.CORE_DCT2, 5),
            synth.Tf(n=4, core=synth.CORE_DCT2, kind=synth.KIND_DENSE, q=np.eye(4)[::-1].copy())]


def test_param_vector_follows_the_layout():
    tfs = table()
    plan = FakePlan(tfs)
    v = T.param_vector(plan).numpy()
    lay = plan._param_layout
    assert v.size == lay[-1] == 23 + 25 + 16        # (8 + 7 + 8) angles, 5 x 5, 4 x 4
    assert np.array_equal(v[lay[0]:lay[1]], tfs[0].angles)
    assert lay[1] == lay[2]                                   # plain core: no entries
    assert np.array_equal(v[lay[2]:lay[3]], tfs[2].q.ravel())
    assert np.array_equal(v[lay[3]:lay[4]], tfs[3].q.ravel())


def test_set_params_keeps_structure_and_places_values():
    tfs = table()
    plan = FakePlan(tfs)
    lay = plan._param_layout
    v = T.param_vector(plan).numpy().copy()
    v[lay[0]:lay[1]] += 0.25
    q = np.linalg.qr(np.random.default_rng(1).standard_normal((5, 5)))[0]
    v[lay[2]:lay[3]] = q.ravel()
    T._set_params(plan, v)
    (new,) = plan.uploads
    for old, d in zip(tfs, new):
        assert (d["n"], d["core"], d["kind"]) == (old.n, old.core, old.kind)
        assert np.array_equal(np.asarray(d["parities"]), np.asarray(old.parities))
    assert np.allclose(new[0]["angles"], tfs[0].angles + 0.25)
    assert "angles" not in new[1] and "q" not in new[1]
    assert np.array_equal(new[2]["q"], q)
    assert new[3]["q"].shape == (4, 4)
    assert np.array_equal(plan._param_values, v)
    # the uploaded table reads back as the same vector
    assert np.array_equal(T.param_vector(plan).numpy(), v)
