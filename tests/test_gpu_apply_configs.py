"""Every H v kernel configuration against the oracle, each pinned in turn
with ed_set_apply_config: the one-kernel variants, the split variants (a
T_up pass, either column blocks staged in shared memory or row gathers one
chunk of columns at a time, then a row pass for the diagonal and T_dn, with
256, 512 or 1024 threads) and the variants whose T_up row chunks a producer
warp stages by TMA, and the multi-vector variants (one row of several
vectors of one sector per thread block), with all their rows-per-block,
pairs-per-thread and occupancy settings.  The 924 x 792 sector gives the row-gather pass a
ragged second chunk (256-pair chunks) and a partly valid second column-pair
group (512-pair chunks).

The sectors put the column pass through each of its layout cases: dim_dn a
multiple of 4 (16-byte pairs, full 4-column blocks), dim_dn = 2 mod 4 (a
2-column tail block), odd dim_dn (element accesses), dim_up not a multiple
of 64 (partial 64-row ELL tiles), dim_up = 1 (no up-spin hops), and a
lattice with many bond classes.  Tolerances as in the other apply tests.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import (LATTICES, torch_cuda, to_dev, from_dev, rel_l2, ed_dtype, max_el,
                      TOL_EL)
from oracle.krylov import make_H

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-13, "c64": 3e-6}

RING10 = synth.ring(10)
RING11 = synth.ring(11)
CASES = [
    ("torus3x4", LATTICES["torus3x4"], 6, 5, 8.0),   # 924 x 792
    ("ring10", RING10, 5, 4, 4.0),                    # 252 x 210 (210 = 2 mod 4)
    ("ring11-odd", RING11, 4, 3, 2.0),                # 330 x 165
    ("ring11-2mod4", RING11, 3, 4, 2.0),              # 165 x 330
    ("ring6-empty-up", LATTICES["ring6"], 0, 3, 2.0), # 1 x 20
    ("complete7", LATTICES["complete7"], 3, 4, 1.3),  # 35 x 35, many classes
]


def configs(ed, dtype):
    want = 1 if dtype == "c128" else 0
    return [c for c in range(ed.ed_apply_config_count())
            if ed.ed_apply_config_info(c)["fp64"] == want]


@pytest.fixture
def pinned(ed_lib):
    yield ed_lib
    ed_lib.ed_set_apply_config(-1)


def test_config_table_has_split_variants_for_both_precisions(ed_lib):
    ed = ed_lib
    for dtype in ("c128", "c64"):
        info = [ed.ed_apply_config_info(c) for c in configs(ed, dtype)]
        assert any(i["split"] for i in info) and any(not i["split"] for i in info)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("name,lat,nu,nd,U", CASES, ids=[c[0] for c in CASES])
def test_every_config_matches_oracle(pinned, dtype, name, lat, nu, nd, U):
    torch = torch_cuda()
    ed = pinned
    A = np.array([0.37, -0.21, 0.0])
    h = ed.Hubbard(lat, nu, nd, U)
    ed.ed_set_field(h.ctx, A)
    v = synth.random_state(h.dim_up, h.dim_dn, seed=5, nvec=2).reshape(2, -1)
    H = make_H(lat, nu, nd, U, A)
    ref = np.stack([H @ v[0], H @ v[1]])
    vd = to_dev(torch, v, dtype)
    for cfg in configs(ed, dtype):
        ed.ed_set_apply_config(cfg)
        wd = torch.full_like(vd, float("nan"))
        if ed.ed_apply_config_info(cfg)["tma"] and h.dim_dn % 2:
            # TMA row chunks need rows of an even number of elements
            with pytest.raises(ed.EDError) as e:
                ed.ed_apply_H(h.ctx, vd, wd, ed_dtype(ed, dtype), nvec=2)
            assert "does not fit" in str(e.value)
            continue
        ed.ed_apply_H(h.ctx, vd, wd, ed_dtype(ed, dtype), nvec=2)
        torch.cuda.synchronize()
        assert ed.ed_get_apply_config(h.ctx)[1] == cfg
        w = from_dev(wd)
        err = rel_l2(w, ref)
        assert err <= TOL[dtype], (cfg, ed.ed_apply_config_info(cfg), err)
        assert max_el(w, ref) <= TOL_EL[dtype], (cfg, max_el(w, ref))
    h.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_split_propagation_with_energy_matches_oracle(pinned, dtype):
    """A short propagation of the 3x4 torus, (6,5), with every split, every
    TMA and every multi-vector configuration of the precision pinned (the
    last with one-vector subgroups): state, <d>, norm and energy (the energy
    runs H v once more per step) against the oracle's trajectory."""
    torch = torch_cuda()
    ed = pinned
    lat = LATTICES["torus3x4"]
    pulse = dict(synth.workload("torus3x4")["pulse_params"], t0=0.1)
    psi0 = synth.complex_normal(924 * 792, 11)
    psi0 /= np.linalg.norm(psi0)
    ref = oracle.propagate(lat, 6, 5, 8.0, psi0, pulse, 0.02, 6, 16, with_energy=True)
    split = [c for c in configs(ed, dtype)
             if any(ed.ed_apply_config_info(c)[k] for k in ("split", "tma", "mv"))]
    for cfg in split:
        ed.ed_set_apply_config(cfg)
        h = ed.Hubbard(lat, 6, 5, 8.0)
        xd = to_dev(torch, psi0, dtype)
        out = ed.ed_propagate(h.ctx, xd, ed_dtype(ed, dtype), pulse, 0.0, 0.02, 6, 16,
                              energy=True)
        torch.cuda.synchronize()
        assert ed.ed_get_apply_config(h.ctx)[0] == cfg
        psi = from_dev(xd)
        h.close()
        if dtype == "c128":
            assert rel_l2(psi, ref["psi"]) <= 1e-10
            assert np.abs(out["docc"] - ref["docc"]).max() <= 1e-10
            assert np.abs(out["energy"] - ref["energy"]).max() <= 1e-10
        else:
            assert rel_l2(psi, ref["psi"]) <= 1e-4
            assert np.abs(out["docc"] - ref["docc"]).max() <= 1e-5
            assert np.abs(out["energy"] - ref["energy"]).max() <= 1e-4


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_multi_vector_configs_with_partial_subgroups(pinned, dtype):
    """Three vectors of one sector under each multi-vector configuration:
    with two or four vectors per thread block the last subgroup is partly
    filled (and with four, all three vectors share one, leaving a slot
    empty).  Element by element against the oracle."""
    torch = torch_cuda()
    ed = pinned
    lat, nu, nd, U = LATTICES["torus3x4"], 6, 5, 8.0
    A = np.array([0.29, 0.13, 0.0])
    h = ed.Hubbard(lat, nu, nd, U)
    ed.ed_set_field(h.ctx, A)
    v = synth.random_state(h.dim_up, h.dim_dn, seed=9, nvec=3).reshape(3, -1)
    H = make_H(lat, nu, nd, U, A)
    ref = np.stack([H @ v[k] for k in range(3)])
    vd = to_dev(torch, v, dtype)
    mv = [c for c in configs(ed, dtype) if ed.ed_apply_config_info(c)["mv"]]
    assert mv
    for cfg in mv:
        ed.ed_set_apply_config(cfg)
        wd = torch.full_like(vd, float("nan"))
        ed.ed_apply_H(h.ctx, vd, wd, ed_dtype(ed, dtype), nvec=3)
        torch.cuda.synchronize()
        assert ed.ed_get_apply_config(h.ctx)[1] == cfg
        w = from_dev(wd)
        assert rel_l2(w, ref) <= TOL[dtype], cfg
        assert max_el(w, ref) <= TOL_EL[dtype], (cfg, max_el(w, ref))
    h.close()
