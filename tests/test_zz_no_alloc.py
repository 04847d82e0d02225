"""frost_accel_noalloc, the entry point for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: for example an application whose allocator owns all
device memory, or time-critical code where an allocation is not allowed. For them the
library offers one entry point that keeps its scratch in a static device array and takes
only caller-owned inputs and outputs. This file calls it through the C-ABI several times in
a row with different sizes (so scratch left by one call cannot leak into the next) and
checks every result against the FP64 oracle on sampled particles and against the
context-based entry point (frost_accel_gradient, mixed precision, the same kernels), with the
mixed-precision tolerance of the other tests: p99.9 of the per-particle relative error
<= 1e-6 and max <= 1e-5. The sizes include the largest one the static array holds, where the
source list has to be split into fewer parts than the context path would use, and a single
particle, whose acceleration is exactly zero. Pytest collects this file last.
"""

import numpy as np
import pytest

import oracle
from paper_2011_14984_gb300 import ics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


def _noalloc(fr, m, x, eps_soft=0.0):
    n = m.shape[0]
    md = torch.as_tensor(m, dtype=torch.float64, device="cuda").contiguous()
    xd = torch.as_tensor(x, dtype=torch.float64, device="cuda").contiguous()
    out = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    fr.frost_accel_noalloc(n, md, xd, 1.0, eps_soft, out, None)
    return out.cpu().numpy()


def _context(fr, m, x, v, eps_soft=0.0):
    f = fr.Frost(m, x, v, precision="mixed", eps_soft=eps_soft)
    a = f.accel_gradient(None, None, want=("acc",))["acc"].cpu().numpy()
    f.close()
    return a


def test_noalloc_matches_the_oracle_and_the_context_entry_point_on_calls_in_a_row():
    assert torch.cuda.is_available(), "needs a CUDA device"
    from paper_2011_14984_gb300 import frost as fr
    fr.load()
    nmax = fr.FROST_NOALLOC_MAX_N
    # other sizes and softenings in a row: a ragged mid size, the largest size the static
    # array holds (its source list split into 4 parts to fit the partials), one particle,
    # and a softened pass
    cases = [(5000, 21, 0.0), (nmax, 23, 0.0), (1, 24, 0.0), (4097, 22, 1e-3)]
    rng = np.random.default_rng(7)
    for n, seed, eps in cases:
        if n == 1:
            m, x = np.array([0.7]), np.array([[0.3, -0.2, 0.1]])
            got = _noalloc(fr, m, x, eps)
            assert np.array_equal(got, np.zeros((1, 3))), got  # no sources: exactly zero
            continue
        m, x, v = ics.plummer(n, seed, masses=ics.kroupa_masses(n, seed))
        got = _noalloc(fr, m, x, eps)
        assert np.isfinite(got).all()
        I = np.sort(rng.choice(n, min(n, 512), replace=False)).astype(np.int32)
        ref = oracle.acc(m, x, I, np.arange(n, dtype=np.int32), eps2=eps * eps)
        e = _rel(got[I], ref)
        assert np.percentile(e, 99.9) <= 1e-6 and e.max() <= 1e-5, (n, np.percentile(e, 99.9), e.max())
        ctx = _context(fr, m, x, v, eps)
        e = _rel(got, ctx)
        assert np.percentile(e, 99.9) <= 1e-6 and e.max() <= 1e-5, (n, np.percentile(e, 99.9), e.max())


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2011_14984_gb300 import frost as fr
    n = fr.FROST_NOALLOC_MAX_N + 1
    m = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    x = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    out = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(fr.FrostError) as e:
        fr.frost_accel_noalloc(n, m, x, 1.0, 0.0, out, None)
    assert e.value.code == fr.FROST_EINVAL
    assert "static scratch" in str(e.value)  # the message of frost_last_error()
    assert float(out.abs().max()) == 0.0  # nothing was launched
