"""Allocation failure, made on the host: a device allocator (the dev_alloc /
dev_free hooks of the configuration) that refuses after a given number of
allocations.  Every refusal comes back as QPIC_ENOMEM, at context creation or
at a particle load, and everything the library did get is returned to the
allocator when the context is destroyed."""
import pytest

import paper_2303_12874_gb300 as q

pytestmark = pytest.mark.gpu


class _Refusing(q._TorchAllocator):
    def __init__(self, grant):
        super().__init__()
        self.grant, self.calls = grant, 0

    def _alloc(self, nbytes, user):
        self.calls += 1
        return 0 if self.calls > self.grant else super()._alloc(nbytes, user)


@pytest.mark.parametrize("grant", [0, 1, 5, 12])
def test_init_reports_enomem_and_returns_everything(grant):
    a = _Refusing(grant)
    with pytest.raises(q.QpicError, match="ENOMEM"):
        q.Sim(64, 16, 0.2, 0.5, torch_alloc=a)
    assert a.calls == grant + 1 and not a.live


def test_load_reports_enomem_and_the_context_survives():
    probe = _Refusing(10 ** 6)
    s = q.Sim(64, 16, 0.2, 0.5, torch_alloc=probe)
    need = probe.calls                       # allocations of a context
    s.close()
    assert not probe.live
    a = _Refusing(need)                      # enough for the context, none for particles
    s = q.Sim(64, 16, 0.2, 0.5, torch_alloc=a)
    with pytest.raises(q.QpicError, match="ENOMEM"):
        s.load_plasma(0.01, 0.0, 0.0, (2, 2, 2))
    s.step(2)                                # fields only: still usable
    s.close()
    assert not a.live
