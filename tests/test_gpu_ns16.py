"""Ns = 16 at half filling: the 4x4 torus sector (8,8), D = 12870^2 =
165,636,900 (2.65 GB per complex128 vector), beyond the paper's CSR memory
limit.  The oracle cannot run a whole Lanczos step at this size, so the
checks use outputs it computes one by one:

* H v on 2,000 sampled elements: w[u,d] = T_up[u,:] . V[:,d] +
  T_dn[d,:] . V[u,:] + U popcount(up_u & dn_d) V[u,d], with the oracle's
  per-spin hopping matrices (Eq. (18) structure, Eqs. (1), (3)).
* U = 0 propagation from one basis configuration (u0, d0): the exact
  midpoint propagator factorises, so every amplitude is a product of two
  8 x 8 determinants of the one-electron midpoint propagators (Cauchy-Binet),
  sampled on 2,000 outputs and on the 200 largest ones.

Tolerances as in the smaller apply and propagation tests.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import synth
from gpu_util import torch_cuda, ed_dtype

pytestmark = pytest.mark.gpu

LAT = synth.lattice_from_name("torus4x4")
N = 8
DIM = 12870


def sample_indices(rng, k):
    return rng.integers(0, DIM, size=k), rng.integers(0, DIM, size=k)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_apply_ns16_half_filling_sampled(ed_lib, dtype, parity_log):
    torch = torch_cuda()
    ed = ed_lib
    A = (0.31, 0.17, 0.0)
    U = 8.0
    h = ed.Hubbard(LAT, N, N, U)
    ed.ed_set_field(h.ctx, A)
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    g = torch.Generator(device="cuda").manual_seed(5)
    vd = torch.randn(h.D, dtype=tdt, device="cuda", generator=g)
    wd = torch.empty_like(vd)
    ed.ed_apply_H(h.ctx, vd, wd, ed_dtype(ed, dtype))
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    us, ds = sample_indices(rng, 2000)
    Tu = oracle.spin_hopping_matrix(LAT, N, A).tocsr()   # = T_dn (n_up = n_dn)
    words = oracle.spin_basis(16, N)
    W = wd.view(DIM, DIM)
    V = vd.view(DIM, DIM)
    # every V entry the sampled outputs need, fetched in one gather
    rows, cols, segs = [], [], []
    for u, d in zip(us, ds):
        ru, rd = Tu.getrow(u), Tu.getrow(d)
        segs.append((ru.data, len(ru.indices), rd.data, len(rd.indices)))
        rows += list(ru.indices) + [u] * len(rd.indices) + [u]
        cols += [d] * len(ru.indices) + list(rd.indices) + [d]
    vals = V[torch.tensor(rows, device="cuda"), torch.tensor(cols, device="cuda")]
    vals = vals.cpu().numpy().astype(np.complex128)
    got = W[torch.from_numpy(us).cuda(), torch.from_numpy(ds).cuda()]
    got = got.cpu().numpy().astype(np.complex128)
    ref = np.zeros(len(us), dtype=np.complex128)
    o = 0
    for k, (u, d) in enumerate(zip(us, ds)):
        du, nu, dd, nd = segs[k]
        diag = U * bin(int(words[u]) & int(words[d])).count("1")
        ref[k] = du @ vals[o:o + nu] + dd @ vals[o + nu:o + nu + nd] + diag * vals[o + nu + nd]
        o += nu + nd + 1
    scale = np.abs(ref).max()
    tol = 1e-13 if dtype == "c128" else 3e-6
    parity_log(f"apply_ns16_sampled_{dtype}", max_el=np.abs(got - ref).max() / scale)
    assert np.abs(got - ref).max() <= tol * scale
    h.close()


def slater_amplitudes(u_up, u_dn, occ_targets_up, occ_targets_dn, occ0_up, occ0_dn):
    a = np.array([np.linalg.det(u_up[np.ix_(o, occ0_up)]) for o in occ_targets_up])
    b = np.array([np.linalg.det(u_dn[np.ix_(o, occ0_dn)]) for o in occ_targets_dn])
    return a * b


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_free_fermion_propagation_ns16_is_slater(ed_lib, dtype, parity_log):
    torch = torch_cuda()
    ed = ed_lib
    pulse = {"A0": 0.9, "omega": 5.0, "sigma": 0.6, "t0": 0.1, "dir": (1.0, 0.7, 0.0)}
    dt, n_steps, m = 0.05, 4, 24
    words = oracle.spin_basis(16, N)
    occ = lambda w: [i for i in range(16) if (int(w) >> i) & 1]  # noqa: E731
    u0, d0 = 1234, 9876
    h = ed.Hubbard(LAT, N, N, 0.0)
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    x = torch.zeros(h.D, dtype=tdt, device="cuda")
    x[u0 * DIM + d0] = 1.0
    ed.ed_propagate(h.ctx, x, ed_dtype(ed, dtype), pulse, 0.0, dt, n_steps, m)
    torch.cuda.synchronize()
    # one-electron midpoint propagator
    u1 = np.eye(16, dtype=np.complex128)
    for n in range(n_steps):
        A = oracle.pulse_A((n + 0.5) * dt, pulse)
        u1 = sla.expm(-1j * dt * oracle.single_particle_matrix(LAT, A)) @ u1
    X = x.view(DIM, DIM)
    rng = np.random.default_rng(3)
    us, ds = sample_indices(rng, 2000)
    # plus the 200 largest amplitudes of the GPU result
    top = torch.topk(x.abs(), 200).indices.cpu().numpy()
    us = np.concatenate([us, top // DIM])
    ds = np.concatenate([ds, top % DIM])
    got = X[torch.from_numpy(us).cuda(), torch.from_numpy(ds).cuda()]
    got = got.cpu().numpy().astype(np.complex128)
    ref = slater_amplitudes(u1, u1, [occ(words[u]) for u in us], [occ(words[d]) for d in ds],
                            occ(words[u0]), occ(words[d0]))
    tol = 1e-10 if dtype == "c128" else 2e-5
    parity_log(f"ns16_slater_{dtype}", amplitude_max_err=np.abs(got - ref).max())
    assert np.abs(ref[-200:]).max() > 1e-3        # the sample sees real amplitudes
    assert np.abs(got - ref).max() <= tol
    h.close()
