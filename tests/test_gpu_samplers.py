"""The parallel samplers side by side (fw_sampler_run, Section 4): DPRS
(Alg. 3), ZPRS (Alg. 4) and the engine's exponential-jump reservoir, at warp
and CTA width, each drawing w_i / sum(w) (Section 4's correctness
propositions).  Independent draws are
tallied against the exact law: total variation and a chi-square test."""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

scipy_stats = pytest.importorskip("scipy.stats")


def _weights(n, kind):
    i = torch.arange(n, dtype=torch.float64)
    if kind == "skew":
        w = 1.0 / (1.0 + i) ** 1.2          # a few heavy entries, a long light tail
    elif kind == "zeros":
        w = (i % 3 != 1).double() * (1.0 + (i % 7))  # every third weight is 0
    else:
        w = 1.0 + (i * 2654435761 % 97) / 97.0
    return w.float()


@pytest.mark.parametrize("method", ["expj", "dprs", "zprs"])
@pytest.mark.parametrize("width", [32, 256])
@pytest.mark.parametrize("n,kind", [(1, "flat"), (7, "skew"), (300, "zeros"), (5000, "skew"), (70000, "flat")])
def test_sampler_law(method, width, n, kind):
    from paper_2404_08364_gb300 import sample
    w = _weights(n, kind)
    reps = 1 << 20
    idx, _ = sample(method, w.cuda(), reps, seed=1234 + n, width=width)
    idx = idx.cpu().numpy()
    assert idx.min() >= 0 and idx.max() < n
    p = (w.double() / w.double().sum()).numpy()
    assert p[idx].min() > 0, "an index of weight 0 was drawn"
    counts = np.bincount(idx, minlength=n).astype(np.float64)
    tv = 0.5 * np.abs(counts / reps - p).sum()
    # pool the cells with small expectations before the chi-square test
    order = np.argsort(p)
    exp = p[order] * reps
    obs = counts[order]
    bins_e, bins_o, acc_e, acc_o = [], [], 0.0, 0.0
    for e, o in zip(exp, obs):
        acc_e += e
        acc_o += o
        if acc_e >= 50:
            bins_e.append(acc_e)
            bins_o.append(acc_o)
            acc_e = acc_o = 0.0
    if acc_e > 0:
        if bins_e:
            bins_e[-1] += acc_e
            bins_o[-1] += acc_o
        else:
            bins_e.append(acc_e)
            bins_o.append(acc_o)
    if len(bins_e) > 1:
        pval = scipy_stats.chisquare(bins_o, bins_e).pvalue
        assert pval > 1e-3, (method, width, n, pval)
    # with 2^20 draws the expected TV of a correct sampler is about
    # sqrt(n_cells / (2 pi reps)); allow a margin
    assert tv < max(2e-3, 1.5 * np.sqrt(n / (2 * np.pi * reps))), (method, width, n, tv)


def test_sampler_all_zero_weights():
    from paper_2404_08364_gb300 import sample
    w = torch.zeros(100, dtype=torch.float32, device="cuda")
    for m in ("expj", "dprs", "zprs"):
        for width in (32, 256):
            idx, _ = sample(m, w, 64, width=width)
            assert (idx == -1).all()
