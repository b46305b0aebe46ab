"""GPU port post-processing against the oracle (Sec. IV: currents impressed on port edges, probe
voltages summed along edges, Z parameters, S parameters with Z0 = 50 Ohm).

* fit_port_rhs: every entry of b against the oracle's -j w (I s) with masked edges zeroed; which
  entries are nonzero must agree exactly (index work).
* fit_probe_voltages: the FP64 sums against the oracle's, to a few ulps of the sum of |terms|.
* fit_z_parameters: Z from one batched GPU solve of every (port, frequency) system against the
  oracle's sparse direct Z.  The solve stops at ||b - A x|| <= tol ||b||, so the bound is
  |Z - Z_direct| <= kappa tol |Z|; on these small lossy grids 1e-6 |Z|max leaves a wide margin at
  tol = 1e-10."""
import numpy as np
import pytest

import fitgen as G
from tests._gpu_util import fitlib, oracle_A, oracle_matrices, torch_cuda

pytestmark = pytest.mark.gpu


def _zcol(case, i, j, k0, k1, sign=1.0):
    nx, ny = case["nx"], case["ny"]
    return [3 * (i + nx * (j + ny * k)) + 2 for k in range(k0, k1)], [sign] * (k1 - k0)


def _three_port_lossy():
    c = G.small_random(8, 7, 6, seed=11, pec_frac=0.0)
    ports = [_zcol(c, 2, 2, 1, 4), _zcol(c, 5, 4, 2, 5), ([3 * (3 + 8 * (3 + 7 * 2)) + 0], [-1.0])]
    return c, ports


def test_port_rhs_matches_oracle():
    """Duplicated edges add, signs flip, masked edges (a low wall plane and PEC cells) stay zero."""
    from oracle import ports as PT
    torch = torch_cuda()
    fit = fitlib()
    case = G.small_random(10, 9, 7, seed=5, pec_frac=0.1)
    nx, ny, nz = 10, 9, 7
    ne = 3 * nx * ny * nz
    _, mask = oracle_A(case, 1.0)
    rng = np.random.default_rng(7)
    edges = rng.integers(0, ne, 300)
    edges = np.concatenate([edges, edges[:40], [3 * (0 + nx * (4 + ny * 3)) + 1]])  # duplicates + a wall edge
    signs = rng.choice([-1.0, 1.0], edges.size)
    assert mask[edges].sum() > 0 and (mask[edges] == 0).sum() > 0
    ws = 2 * np.pi * np.array([0.7e9, 3e9, 11e9])
    cur = 0.37
    with fit.Grid.from_case(case) as g:
        b = torch.full((len(ws) * ne,), 5.0 + 5.0j, dtype=torch.complex128, device="cuda")  # overwritten
        fit.fit_port_rhs(g.h, ws, edges, signs, b, current=cur)
        torch.cuda.synchronize()
        got = b.cpu().numpy().reshape(len(ws), ne)
    for f, w in enumerate(ws):
        want = PT.port_rhs(w, ne, edges, signs, mask, current=cur)
        assert np.array_equal(got[f] != 0, want != 0), f
        assert np.all(got[f].real == 0)
        assert np.allclose(got[f], want, rtol=1e-15, atol=0), f


def test_port_rhs_empty_port_zeroes_b():
    torch = torch_cuda()
    fit = fitlib()
    case = G.small_random(5, 4, 3, seed=2)
    ne = 3 * 5 * 4 * 3
    with fit.Grid.from_case(case) as g:
        b = torch.ones(2 * ne, dtype=torch.complex128, device="cuda")
        fit.fit_port_rhs(g.h, [1e9, 2e9], [], [], b)
        torch.cuda.synchronize()
        assert int(torch.count_nonzero(b)) == 0


def test_probe_voltages_match_oracle():
    """Probes of 0, 1, 3, 257 and 1500 edges (the last two span several strides of the 256-thread CTA),
    with repeated edges, over a batch of 3 systems."""
    from oracle import ports as PT
    torch = torch_cuda()
    fit = fitlib()
    case = G.small_random(12, 11, 10, seed=9)
    ne = 3 * 12 * 11 * 10
    rng = np.random.default_rng(3)
    probes = []
    for n in (0, 1, 3, 257, 1500):
        e = rng.integers(0, ne, n)
        probes.append((e, rng.choice([-1.0, 1.0], n)))
    x = G.random_vector(ne, 21, batch=3)
    with fit.Grid.from_case(case) as g:
        xd = torch.from_numpy(np.ascontiguousarray(x.reshape(-1))).cuda()
        V = fit.fit_probe_voltages(g.h, xd, probes)
    assert V.shape == (3, len(probes))
    for f in range(3):
        for q, (e, s) in enumerate(probes):
            want = PT.probe_voltage(x[f], e, s)
            scale = np.sum(np.abs(x[f][e])) if len(e) else 0.0
            assert abs(V[f, q] - want) <= 1e-14 * scale, (f, q, V[f, q], want)
    assert V[0, 0] == 0


def test_probe_voltages_are_deterministic():
    torch = torch_cuda()
    fit = fitlib()
    case = G.small_random(12, 11, 10, seed=9)
    ne = 3 * 12 * 11 * 10
    rng = np.random.default_rng(4)
    probes = [(rng.integers(0, ne, 2000), rng.choice([-1.0, 1.0], 2000))]
    x = G.random_vector(ne, 22)
    with fit.Grid.from_case(case) as g:
        xd = torch.from_numpy(x).cuda()
        v0 = fit.fit_probe_voltages(g.h, xd, probes)
        for _ in range(3):
            assert np.array_equal(fit.fit_probe_voltages(g.h, xd, probes), v0)


@pytest.mark.parametrize("method,precision", [(0, 0), (0, 1), (1, 1), (2, 1)])
def test_z_parameters_three_port_lossy(method, precision):
    """The 3-port lossy network of the oracle's pins, at two frequencies in one batch of 6 systems."""
    from oracle import ports as PT
    torch_cuda()
    fit = fitlib()
    case, ports = _three_port_lossy()
    ws = 2 * np.pi * np.array([1e9, 3e9])
    with fit.Grid.from_case(case) as g:
        st, Z, rep = fit.fit_z_parameters(g.h, ws, ports, 1e-10, current=2.0, method=method, precision=precision,
                                          max_iter=20000, max_outer=1000)
    assert st == 0, rep
    assert len(rep) == 6 and all(r["status"] == 0 and r["relres"] <= 1e-10 for r in rep)
    for f, w in enumerate(ws):
        A, mask = oracle_A(case, w)
        Zo = PT.z_matrix(A.tocsr(), w, ports, mask)
        assert np.abs(Z[f] - Zo).max() <= 1e-6 * np.abs(Zo).max(), (f, Z[f], Zo)
        assert np.abs(Z[f] - Z[f].T).max() <= 1e-6 * np.abs(Zo).max()  # reciprocity
        S = fit.fit_z_to_s(Z[f])
        assert np.abs(S - PT.z_to_s(Zo)).max() <= 1e-5
        assert np.linalg.norm(S, 2) <= 1 + 1e-6  # passive


def test_z_parameters_masked_port_gives_a_zero_column():
    """A port lying in the low x wall (all its edges masked) drives nothing: b = 0, the solve returns
    x = 0 at once, and its Z column and row vanish; the other port is unaffected."""
    from oracle import ports as PT
    torch_cuda()
    fit = fitlib()
    case, ports = _three_port_lossy()
    nx, ny = case["nx"], case["ny"]
    wall = ([3 * (0 + nx * (3 + ny * k)) + 2 for k in (1, 2)], [1.0, 1.0])  # z-edges in the plane i = 0
    w = 2 * np.pi * 2e9
    with fit.Grid.from_case(case) as g:
        st, Z, rep = fit.fit_z_parameters(g.h, [w], [ports[0], wall], 1e-10)
    assert st == 0 and rep[1]["iterations"] == 0
    assert Z[0, 0, 1] == 0 and Z[0, 1, 1] == 0  # x = 0 exactly when the wall port is driven
    A, mask = oracle_A(case, w)
    Zo = PT.z_matrix(A.tocsr(), w, [ports[0]], mask)
    assert abs(Z[0, 1, 0]) <= 1e-12 * abs(Zo[0, 0])  # masked rows are the identity with b = 0 there
    assert abs(Z[0, 0, 0] - Zo[0, 0]) <= 1e-6 * abs(Zo[0, 0])


def test_z_parameters_rejects_bad_ports():
    torch_cuda()
    fit = fitlib()
    case, ports = _three_port_lossy()
    ne = 3 * 8 * 7 * 6
    with fit.Grid.from_case(case) as g:
        with pytest.raises(fit.FitError):
            fit.fit_z_parameters(g.h, [1e9], [([ne], [1.0])], 1e-8)
        with pytest.raises(fit.FitError):
            fit.fit_z_parameters(g.h, [1e9], ports, 1e-8, current=0.0)


def test_port_rhs_and_probes_full_size():
    """layered128 at full size: four 8-edge z-column ports at two frequencies.  b is checked on every port
    edge and on sampled other edges; probe sums of a random device vector against the oracle's."""
    from oracle import ports as PT
    torch = torch_cuda()
    fit = fitlib()
    case = G.layered_blocks()
    nx, ny, nz = 128, 128, 128
    ne = 3 * nx * ny * nz
    _, _, _, mask = oracle_matrices(case)
    ports = [_zcol(case, i, j, 0, 8) for i, j in ((20, 90), (76, 68), (92, 39), (99, 48))]
    ws = 2 * np.pi * np.array([1e9, 3e9])
    rng = np.random.default_rng(8)
    others = rng.choice(ne, 500, replace=False)
    with fit.Grid.from_case(case) as g:
        b = torch.empty(len(ws) * ne, dtype=torch.complex128, device="cuda")
        for e, s in ports:
            fit.fit_port_rhs(g.h, ws, e, s, b, current=1.0)
            torch.cuda.synchronize()
            idx = np.unique(np.concatenate([np.asarray(e), others]))
            for f, w in enumerate(ws):
                got = b[f * ne + torch.from_numpy(idx).cuda()].cpu().numpy()
                want = PT.port_rhs(w, ne, e, s, mask)[idx]
                assert np.allclose(got, want, rtol=1e-15, atol=0)
        gen = torch.Generator(device="cuda")
        gen.manual_seed(3)
        x = torch.randn(2 * ne, dtype=torch.complex128, device="cuda", generator=gen)
        V = fit.fit_probe_voltages(g.h, x, ports)
        for f in range(2):
            for q, (e, s) in enumerate(ports):
                xe = x[f * ne + torch.tensor(e, device="cuda")].cpu().numpy()
                xf = np.zeros(ne, np.complex128)
                xf[e] = xe
                want = PT.probe_voltage(xf, e, s)
                assert abs(V[f, q] - want) <= 1e-14 * np.sum(np.abs(xe))
