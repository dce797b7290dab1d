"""rt_tail_prior (CUDA) against the FP64 reference of the specular tail prior."""
import numpy as np
import pytest

from oracle import prior as P

pytestmark = pytest.mark.gpu


def _run(rates, air, level, n_nodes, t0, dt, n_bins):
    import torch
    from paper_1811_05784_gb300 import rt
    dev = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda")
    out = rt.rt_tail_prior(dev(rates), dev(air), dev(level), n_nodes, t0, dt, n_bins)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n_nodes,n_bins", [(40, 300), (64, 195), (1, 7), (33, 257)])
def test_prior_matches_reference(n_nodes, n_bins):
    """Several 1024-direction chunks with a ragged last one, bin blocks of 256
    with a ragged tail, zero rates and zero air.  FP32 evaluates exp(-R t)
    with R and t rounded to float: relative error <= (R t + 4) 2^-22 < 1e-4 for
    every value above 1e-30 of the level; smaller values agree in absolute
    terms."""
    g = np.random.default_rng(n_nodes * 1000 + n_bins)
    n = 5
    rates = g.uniform(0.5, 300.0, (n, 3, 8)).astype(np.float32)
    rates[1, 0] = 0.0                      # an axis without absorption
    rates[2] = 0.0                         # no walls absorb: air alone
    air = g.uniform(0.0, 3.0, (n, 8)).astype(np.float32)
    air[0] = 0.0
    air[2, 0] = 0.0                        # no loss at all in one band: flat curve
    level = g.uniform(1e-6, 1e-2, n).astype(np.float32)
    t0, dt = 0.05, 0.01
    got = _run(rates, air, level, n_nodes, t0, dt, n_bins)
    ref = P.tail_prior(rates.astype(np.float64), air.astype(np.float64), level.astype(np.float64), n_nodes,
                       np.float64(np.float32(t0)), np.float64(np.float32(dt)), n_bins)
    big = ref > 1e-30 * level[:, None, None]
    assert big.sum() > 0.3 * big.size
    rel = np.abs(got[big] / ref[big] - 1)
    assert rel.max() < 1e-4, rel.max()
    small = ~big
    assert np.all(np.abs(got[small] - ref[small]) <= 1e-30 * np.broadcast_to(level[:, None, None], ref.shape)[small])
    if n_nodes >= 8:                       # the rule's weights sum to 1: no loss keeps the level
        assert np.allclose(got[2, 0], level[2], rtol=1e-6)


def test_prior_rejects_bad_arguments():
    import torch
    from paper_1811_05784_gb300 import rt
    x = torch.zeros((1, 3, 8), device="cuda")
    a = torch.zeros((1, 8), device="cuda")
    lv = torch.ones(1, device="cuda")
    for kw in (dict(n_nodes=0), dict(n_nodes=257), dict(dt=0.0), dict(t0=-1.0), dict(n_bins=0)):
        args = dict(n_nodes=8, t0=0.0, dt=0.01, n_bins=10)
        args.update(kw)
        with pytest.raises(rt.RtError):
            rt.rt_tail_prior(x, a, lv, args["n_nodes"], args["t0"], args["dt"], args["n_bins"],
                             out=torch.empty((1, 8, max(args["n_bins"], 1)), device="cuda"))
