"""Full-size assembly parity on sampled outputs: the Q1 cube (64^3, 2.1M points) and the P2-tet strip
(48^3 x 6, 7.3M points) at a seeded iterate and state, in the launch configuration of the load path.

The oracle cannot assemble the whole matrix at these sizes, but a row of K (and an entry of F) only
receives contributions from the elements that contain its node: for a seeded sample of nodes the
oracle assembles the sub-mesh of those elements, with the same displacements and state, and its rows
for the sampled nodes must equal the GPU's rows (1e-11 relative, both forms of the tangent); the
plastic flags of the sub-mesh's points must be identical.
"""
import numpy as np
import pytest

from oracle import constitutive as OC
from oracle.fem import Assembler, Geometry
from synthetic import DP, p2_tet_strip_dp, q1_cube_vm
from synthetic.random_states import random_displacement, random_state

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = 1e-11


@pytest.fixture(scope="module")
def ep():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_04155_gb300 import build as b
    b.build()
    import paper_1805_04155_gb300.ep as mod
    return mod


def _iterate(prob, n_int, seed):
    """Seeded displacement and state giving a mix of elastic and plastic points (as the small
    fed-iterate tests: strains of a few 1e-3, plastic strains of 3e-4)."""
    m = prob.mesh
    nc = OC.n_comp(m.dim)
    u = random_displacement(m.coords, prob.dirichlet, 2.5e-3 * 10.0 / max(m.shape), seed, affine=max(m.shape) * 0.1)
    if prob.material.model == DP:
        u = u + 1.0e-3 * m.coords.ravel() * (1 - prob.dirichlet)
    ep_, alpha = random_state(n_int, nc, 3e-4, seed + 1, hard_scale=1e-3)
    return u, ep_, alpha


@pytest.mark.parametrize("make", [lambda: q1_cube_vm(), lambda: p2_tet_strip_dp()], ids=["q1_cube_64", "p2_tet_48"])
def test_full_size_assembly_sampled_rows(ep, make):
    prob = make()
    m = prob.mesh
    dim = m.dim
    ctx = ep.Context.from_problem(prob)
    info = ctx.info
    n_q, n_p = info.n_q, info.n_p
    u, ep_, hard = _iterate(prob, info.n_int, seed=7)
    ctx.set(ep.EP_PLASTIC_STRAIN, ep_)
    ctx.set(ep.EP_HARDENING, hard)
    rng = np.random.default_rng(8)
    sample = np.unique(np.concatenate([rng.choice(m.n_nodes, 60, replace=False), [0, m.n_nodes - 1]]))
    # sub-mesh: every element holding a sampled node
    sub_e = np.nonzero(np.isin(m.elem, sample).any(axis=1))[0]
    sub_nodes, local = np.unique(m.elem[sub_e], return_inverse=True)
    sub_elem = local.reshape(len(sub_e), n_p).astype(np.int32)
    sub_coords = m.coords[sub_nodes]
    ips = (sub_e[:, None] * n_q + np.arange(n_q)[None, :]).ravel()
    sub_u = u.reshape(-1, dim)[sub_nodes].ravel()
    g = Geometry(sub_coords, sub_elem, m.elem_type, dim)
    K_b, G_b = OC.moduli(prob.material.E, prob.material.nu)
    C = OC.elastic_tangent(K_b, G_b)
    asm = Assembler(g, C)
    hard_sub = hard[..., ips]
    res = OC.constitutive(prob.material, dim, g.strain(asm.B, sub_u), ep_[:, ips], hard_sub)
    F_or = asm.internal_force(res["S_in"])
    rows_local = np.searchsorted(sub_nodes, sample)
    rp = ctx.get(ep.EP_K_ROW_PTR)
    ci = ctx.get(ep.EP_K_COL_IDX)
    blocks = np.concatenate([np.arange(rp[n], rp[n + 1]) for n in sample])
    vals_dev = torch.empty((info.nnz_blocks, dim, dim), dtype=torch.float64, device="cuda")
    for split in (True, False):
        n_pl = ctx.assemble(u, split=split)
        assert 0 < n_pl < info.n_int
        F = ctx.get(ep.EP_F_INT).reshape(-1, dim)
        F_sub = F_or.reshape(-1, dim)[rows_local]
        e_F = np.abs(F[sample] - F_sub).max() / np.abs(F_sub).max()
        ctx.get(ep.EP_K_VALUES, out=vals_dev)
        vals = vals_dev[torch.from_numpy(blocks).cuda()].cpu().numpy()
        K_or = (asm.tangent_split(res["DS_in"]) if split else asm.tangent_full(res["DS_in"])).tocsr()
        err = scale = 0.0
        k = 0
        for n, rl in zip(sample, rows_local):
            cols = ci[rp[n]:rp[n + 1]]
            cl = np.searchsorted(sub_nodes, cols)
            assert np.array_equal(sub_nodes[cl], cols)      # every neighbour lies in the sub-mesh
            for a in range(dim):
                row_or = K_or[rl * dim + a].toarray().ravel().reshape(-1, dim)
                gpu = np.zeros_like(row_or)
                gpu[cl] = vals[k:k + len(cols), a, :]
                err = max(err, np.abs(gpu - row_or).max())
                scale = max(scale, np.abs(row_or).max())
                # nothing outside the pattern: the oracle row vanishes off the node's neighbours
                mask = np.ones(row_or.shape[0], dtype=bool)
                mask[cl] = False
                assert np.all(row_or[mask] == 0.0)
            k += len(cols)
        print(f"\n{prob.name} split={split}: {len(sample)} sampled nodes, {len(sub_e)} elements, "
              f"{int(res['plastic'].astype(bool).sum())}/{len(ips)} plastic points; K rows rel err {err / scale:.2e}, "
              f"F rel err {e_F:.2e}")
        assert err / scale < TOL and e_F < TOL
    assert 0 < int(res["plastic"].astype(bool).sum()) < len(ips)   # both regimes in the sample
    # commit: flags, stress and plastic strain of the sampled points
    ctx.commit(u)
    assert np.array_equal(ctx.get(ep.EP_PLASTIC_FLAG)[ips], res["plastic"].astype(np.uint8))
    e_s = np.abs(ctx.get(ep.EP_STRESS)[:, ips] - res["S"]).max() / np.abs(res["S"]).max()
    e_p = np.abs(ctx.get(ep.EP_PLASTIC_STRAIN)[:, ips] - res["ep"]).max() / np.abs(res["ep"]).max()
    print(f"commit: stress rel err {e_s:.2e}, plastic strain rel err {e_p:.2e}")
    assert e_s < TOL and e_p < TOL
    ctx.close()
