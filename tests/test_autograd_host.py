"""The torch.autograd wrapper of the Greeks call, on the CPU with the library
call replaced by a fake of known derivatives: the options it passes, the
prices it returns and the chain rule of its backward pass."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def amc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1205_0106_gb300 as amc
    return amc


def test_american_price_forward_and_backward(amc, monkeypatch):
    import torch
    from paper_1205_0106_gb300.autograd import american_price
    seen = []

    def fake_greeks(ctx, opts, prec):
        seen.append((ctx, opts, prec))
        S = np.array([o["S0"] for o in opts])
        sg = np.array([o["sigma"] for o in opts])
        K = np.array([o["K"] for o in opts])
        return S * S * sg - K, 2 * S * sg, S * S                  # price, d/dS0, d/dsigma

    monkeypatch.setattr(amc, "amc_greeks", fake_greeks)
    S0 = torch.tensor([36.0, 40.0, 44.0], dtype=torch.float64, requires_grad=True)
    sig = torch.tensor([0.2, 0.3, 0.4], dtype=torch.float64, requires_grad=True)
    p = american_price("ctx", S0, sig, K=[40.0, 41.0, 42.0], r=0.06, T=1.0, n_steps=50, n_paths=4096, seed=7,
                       prec=amc.AMC_FP64)
    ctx, opts, prec = seen[0]
    assert ctx == "ctx" and prec == amc.AMC_FP64 and len(opts) == 3
    assert [o["K"] for o in opts] == [40.0, 41.0, 42.0] and all(o["n_steps"] == 50 and o["seed"] == 7 for o in opts)
    assert [o["S0"] for o in opts] == [36.0, 40.0, 44.0] and [o["sigma"] for o in opts] == [0.2, 0.3, 0.4]
    torch.testing.assert_close(p, (S0 * S0 * sig - torch.tensor([40.0, 41.0, 42.0], dtype=torch.float64)).detach())
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64)
    (p * w).sum().backward()
    torch.testing.assert_close(S0.grad, w * 2 * S0.detach() * sig.detach())
    torch.testing.assert_close(sig.grad, w * S0.detach() ** 2)


def test_american_price_checks_its_arguments(amc):
    import torch
    from paper_1205_0106_gb300.autograd import american_price
    with pytest.raises(ValueError):
        american_price(None, torch.ones(3, dtype=torch.float64), torch.ones(2, dtype=torch.float64), 40.0, 0.06,
                       1.0, 10, 100)
    with pytest.raises(ValueError):
        american_price(None, torch.ones(3, dtype=torch.float64), torch.ones(3, dtype=torch.float64), [40.0, 41.0],
                       0.06, 1.0, 10, 100)
