"""Host-side logic of the autograd binding (no GPU): quad strengths are
substituted in lattice order, per-bunch strengths become per_bunch_k
columns, and a strength vector of the wrong length is rejected."""
import numpy as np
import pytest

from paper_2402_17248_gb300.grad import _with_strengths
from synth import lattice


def test_strengths_substituted_in_order():
    els = lattice.staged_beamline(2, 10)
    nq = sum(e["kind"] == "quad" for e in els)
    k = np.arange(1.0, nq + 1.0)
    out = _with_strengths(els, k)
    assert [e["k"] for e in out if e["kind"] == "quad"] == list(k)
    assert [e["k"] for e in els if e["kind"] == "quad"] != list(k)  # input not modified
    assert all(a["kind"] == b["kind"] for a, b in zip(els, out))


def test_per_bunch_strengths_become_columns():
    els = lattice.staged_beamline(1, 10)
    nq = sum(e["kind"] == "quad" for e in els)
    k = np.arange(3.0 * nq).reshape(3, nq)
    out = _with_strengths(els, k)
    cols = [e["per_bunch_k"] for e in out if e["kind"] == "quad"]
    for q, c in enumerate(cols):
        assert np.array_equal(c, k[:, q])


def test_wrong_length_rejected():
    els = lattice.staged_beamline(1, 10)
    with pytest.raises(ValueError):
        _with_strengths(els, np.zeros(3))
