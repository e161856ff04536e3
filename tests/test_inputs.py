"""The seeded synthetic workloads (no GPU): the serving stream and the
batched uneven workload have the distributions their docstrings state, the
Fourier right-hand sides equal their closed forms, and the generators are
reproducible."""
import numpy as np

from paper_2504_10710_gb300 import inputs


def test_serving_stream_distribution():
    meshes, reqs = inputs.serving_stream(nreq=2000, rate=200.0)
    assert len(meshes) == 24 and len(reqs) == 2000
    d2 = [m for m in meshes if m.dim == 2]
    d3 = [m for m in meshes if m.dim == 3]
    assert len(d2) == 16 and len(d3) == 8
    for m in d2:
        assert 4 <= m.nelem[0] <= 64 and m.nelem[0] == m.nelem[1] and 4 <= m.order <= 12
        assert 0.0 <= m.params["amp"] <= 0.2 and m.nrhs == 4
    for m in d3:
        assert 8 <= m.nelem[0] <= 32 and len(set(m.nelem)) == 1 and 4 <= m.order <= 8
    # the top of the 3-D range is in the pool
    assert any(m.nelem == (32, 32, 32) and m.order == 8 for m in d3)
    t = np.array([r[0] for r in reqs])
    assert np.all(np.diff(t) > 0)
    # Poisson arrivals: mean gap 1/200 s within 10 % for 2000 samples
    assert abs(np.mean(np.diff(t)) - 1 / 200.0) < 0.1 / 200.0
    kinds = np.array([meshes[mi].dim for _, mi, _ in reqs])
    assert (kinds == 2).sum() == 1000 and (kinds == 3).sum() == 1000
    assert all(0 <= ri < meshes[mi].nrhs for _, mi, ri in reqs)
    # reproducible
    m2, r2 = inputs.serving_stream(nreq=2000, rate=200.0)
    assert r2 == reqs and [m.name for m in m2] == [m.name for m in meshes]


def test_batch_uneven_distribution():
    ws = inputs.batch_uneven()
    assert len(ws) == 256
    n = np.array([w.nelem[0] for w in ws])
    p = np.array([w.order for w in ws])
    assert n.min() >= 4 and n.max() <= 64 and p.min() >= 4 and p.max() <= 12
    assert all(w.nelem[0] == w.nelem[1] for w in ws)
    dof = sum(w.ndof() for w in ws)
    assert 20e6 < dof < 33e6


def test_fourier_rhs_matches_its_closed_form():
    f3, par3 = inputs.fourier_rhs_3d(inputs.rng_for(9, 3))
    f2, par2 = inputs.fourier_rhs_2d(inputs.rng_for(9, 4))
    x, y, z = np.random.default_rng(3).uniform(-0.3, 1.3, (3, 7, 9, 11))
    ref3 = sum(a * np.sin(np.pi * k[0] * x) * np.sin(np.pi * k[1] * y) * np.sin(np.pi * k[2] * z)
               for a, k in zip(par3["a"], par3["k"]))
    ref2 = sum(a * np.sin(np.pi * m * x) * np.sin(np.pi * n * y) for a, m, n in zip(par2["a"], par2["m"], par2["n"]))
    assert np.abs(f3(x, y, z) - ref3).max() < 1e-12 * max(1.0, np.abs(ref3).max())
    assert np.abs(f2(x, y) - ref2).max() < 1e-12 * max(1.0, np.abs(ref2).max())
    # scalars and chunk boundaries (more nodes than one evaluation chunk)
    assert abs(float(f2(0.3, 0.4)) - sum(a * np.sin(np.pi * m * 0.3) * np.sin(np.pi * n * 0.4)
                                         for a, m, n in zip(par2["a"], par2["m"], par2["n"]))) < 1e-12
    big = np.linspace(0.0, 1.0, (1 << 20) + 37)
    v = f2(big, 0.5 * big)
    i = np.array([0, 1 << 19, (1 << 20) - 1, 1 << 20, (1 << 20) + 36])
    ref = sum(a * np.sin(np.pi * m * big[i]) * np.sin(np.pi * n * 0.5 * big[i])
              for a, m, n in zip(par2["a"], par2["m"], par2["n"]))
    assert np.abs(v[i] - ref).max() < 1e-12
