"""Failure handling with host-injected faults (SWGB_FAULT): a failed device
allocation or a failed copy returns its status through the C ABI, frees what
was allocated, and leaves the context usable.  Nothing faults the GPU: the
named step reports an error instead of running."""
import numpy as np
import pytest

from helpers import oracle_all, seqset
from paper_2309_09609_gb300 import build as nvbuild
from paper_2309_09609_gb300 import swgb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    nvbuild.build()
    swgb.lib()


def test_allocation_and_copy_faults_return_status_and_the_context_survives(monkeypatch):
    rng = np.random.default_rng(40)
    db = seqset(rng, list(rng.integers(1, 500, size=200)) + [2500])
    q = seqset(rng, [40, 300])
    want = oracle_all(q, db)

    monkeypatch.setenv("SWGB_FAULT", "alloc")
    with pytest.raises(swgb.SwError) as e:
        swgb.Database.from_seqset(db)
    assert e.value.status == swgb.SW_ENOMEM
    monkeypatch.delenv("SWGB_FAULT")
    d = swgb.Database.from_seqset(db)

    monkeypatch.setenv("SWGB_FAULT", "alloc")
    with pytest.raises(swgb.SwError) as e:
        d.plan(2, 1000)
    assert e.value.status == swgb.SW_ENOMEM
    with pytest.raises(swgb.SwError) as e:
        d.search(q.res, q.lens)                      # the one-shot search's own plan
    assert e.value.status == swgb.SW_ENOMEM
    monkeypatch.delenv("SWGB_FAULT")
    p = d.plan(2, 1000)

    monkeypatch.setenv("SWGB_FAULT", "copy")
    with pytest.raises(swgb.SwError) as e:
        p.search(q.res, q.lens)
    assert e.value.status == swgb.SW_ECUDA and "injected" in str(e.value)
    monkeypatch.delenv("SWGB_FAULT")
    assert (p.search(q.res, q.lens) == want).all()   # the same plan, still usable
    assert (d.search(q.res, q.lens) == want).all()
