"""The seeded input generators: determinism, CSR invariants, recipe facts."""

import pytest
import torch

import fw_inputs as fi


def _check_csr(g):
    rp, col = g.row_ptr, g.col.to(torch.int64)
    assert rp[0] == 0 and rp[-1] == g.m and (rp[1:] >= rp[:-1]).all()
    src = torch.repeat_interleave(torch.arange(g.n), rp[1:] - rp[:-1])
    assert (src != col).all()                      # no self loops
    key = src * g.n + col
    assert (key[1:] > key[:-1]).all()              # rows sorted, no duplicates
    # symmetric with equal attributes in both directions
    rkey = col * g.n + src
    order = torch.argsort(rkey)
    assert torch.equal(rkey[order], key)
    assert torch.equal(g.w_u32[order], g.w_u32)
    if g.etype is not None:
        assert torch.equal(g.etype[order], g.etype)


def test_chung_lu_recipe():
    g = fi.chung_lu()
    _check_csr(g)
    assert g.n == 1000
    assert 5000 <= g.m // 2 <= 10000
    w = g.w_u32
    assert int(w.min()) >= 1 and int(w.max()) <= 5
    assert torch.equal(g.w_f32, w.to(torch.float32))
    assert g.manifest() == fi.chung_lu().manifest()


def test_rmat_recipe_and_chunk_independence():
    g = fi.rmat(10, types_seed=2)
    _check_csr(g)
    h = fi.rmat(10, types_seed=2, chunk=1000)
    assert torch.equal(g.col, h.col) and torch.equal(g.row_ptr, h.row_ptr)
    assert torch.equal(g.etype, h.etype)
    wu = g.w_u32.to(torch.int64)
    assert int(wu.min()) >= 16384 and int(wu.max()) < 81920
    assert torch.equal(g.w_f32.to(torch.float64) * 16384, wu.to(torch.float64))
    assert set(g.etype.unique().tolist()) == {0, 1, 2, 3, 4}
    d = g.degrees()
    assert int(d.argmax()) == 0  # unpermuted R-MAT: vertex 0 is the top hub


def test_starts_and_lengths():
    s = fi.random_starts(1000, 5000, 7)
    assert int(s.min()) >= 0 and int(s.max()) < 1000
    assert torch.equal(s, fi.random_starts(1000, 5000, 7))
    ln = fi.uniform_lengths(5000, 10, 80, 3)
    assert int(ln.min()) == 10 and int(ln.max()) == 80


@pytest.mark.parametrize("sigma", [1, 3])
def test_lognormal_weights(sigma):
    """log w has mean 0 and standard deviation sigma (Appendix C.1's weights);
    the integer weight is at least 1 and the float is it times 2^-14."""
    g = fi.rmat(12, weights=f"lognormal{sigma}")
    wu = g.w_u32.to(torch.int64)
    assert int(wu.min()) >= 1
    lw = torch.log(wu.double() / 16384.0)
    assert abs(float(lw.mean())) < 0.05
    assert abs(float(lw.std()) - sigma) < 0.05 * sigma
    rel = (g.w_f32.double() - wu.double() / 16384.0).abs() / (wu.double() / 16384.0)
    assert float(rel.max()) <= 2.0 ** -24
