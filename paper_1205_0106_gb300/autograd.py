"""Option prices as differentiable functions of spot and volatility.

``american_price`` returns the prices of n options as a tensor; its gradient
with respect to ``S0`` and ``sigma`` is the frozen-boundary pathwise delta
and vega that the library's sweep computes in the same pass as the price
(``amc_greeks``): the exercise dates tau of each path are held fixed and the
discounted payoff e^{-r t_tau} h(S_tau) is differentiated along the path,
dS_tau/dS0 = S_tau / S0 and dS_tau/dsigma = S_tau (W_tau - sigma t_tau).
The forward pass is one library call; the backward pass multiplies the
incoming gradient by the saved delta and vega.  With S0 and sigma on a CUDA
device the call is amc_greeks_device on PyTorch's current stream: spot and
volatility are read from the tensors on the GPU and the results are written
into GPU tensors, with no host round trip and no synchronisation (an
invalid spot or volatility gives NaN for that option).  CPU tensors take the
blocking host call.  Argument marshalling only: the prices and their
derivatives come from the CUDA kernels.
"""
import torch

from . import AMC_MIXED, AMC_PUT, AMC_RULE_LSM


class AmericanPrice(torch.autograd.Function):
    """prices = f(S0, sigma) for the options described by ``fixed`` (one
    dict per option with K, r, T, n_steps, n_paths, basis, type, seed,
    rule); S0 and sigma are 1-D tensors of the same length."""

    @staticmethod
    def forward(ctx, S0, sigma, fixed, amc_ctx, prec):
        import paper_1205_0106_gb300 as pkg
        if S0.is_cuda:
            dev = S0.device
            s0 = S0.detach().to(torch.float64).contiguous()
            sg = sigma.detach().to(device=dev, dtype=torch.float64).contiguous()
            p, d, v = (torch.empty(s0.shape[0], dtype=torch.float64, device=dev) for _ in range(3))
            opts = [dict(o, S0=1.0, sigma=1.0) for o in fixed]     # not read: spot and volatility come from s0, sg
            pkg.amc_greeks_device(amc_ctx, opts, p, d, v, prec, S0=s0, sigma=sg,
                                  stream=torch.cuda.current_stream(dev))
            ctx.save_for_backward(d.to(S0.dtype), v.to(sigma.dtype))
            return p.to(S0.dtype)
        s0 = S0.detach().to("cpu", torch.float64).tolist()
        sg = sigma.detach().to("cpu", torch.float64).tolist()
        opts = [dict(o, S0=a, sigma=b) for o, a, b in zip(fixed, s0, sg)]
        p, d, v = pkg.amc_greeks(amc_ctx, opts, prec)
        ctx.save_for_backward(torch.as_tensor(d, dtype=S0.dtype, device=S0.device),
                              torch.as_tensor(v, dtype=sigma.dtype, device=sigma.device))
        return torch.as_tensor(p, dtype=S0.dtype, device=S0.device)

    @staticmethod
    def backward(ctx, grad):
        delta, vega = ctx.saved_tensors
        return grad * delta, grad * vega, None, None, None


def american_price(amc_ctx, S0, sigma, K, r, T, n_steps, n_paths, basis=3, type=AMC_PUT, seed=0, rule=AMC_RULE_LSM,
                   prec=AMC_MIXED):
    """Prices of n options (the Longstaff-Schwartz or European rule, which
    have frozen-boundary Greeks).  S0 and sigma are tensors of shape [n] (or
    scalars, n = 1); every other argument is a scalar shared by the options
    or a sequence of length n."""
    S0 = torch.atleast_1d(torch.as_tensor(S0, dtype=torch.float64))
    sigma = torch.atleast_1d(torch.as_tensor(sigma, dtype=torch.float64, device=S0.device))
    if S0.dim() != 1 or S0.shape != sigma.shape:
        raise ValueError("S0 and sigma must be 1-D tensors of one length")
    n = S0.shape[0]

    def each(x):
        if isinstance(x, (list, tuple)) or (hasattr(x, "__len__") and not isinstance(x, str)):
            if len(x) != n:
                raise ValueError("per-option arguments must have length %d" % n)
            return list(x)
        return [x] * n

    cols = {k: each(v) for k, v in dict(K=K, r=r, T=T, n_steps=n_steps, n_paths=n_paths, basis=basis, type=type,
                                        seed=seed, rule=rule).items()}
    fixed = [{k: cols[k][i] for k in cols} for i in range(n)]
    for o in fixed:
        o["K"], o["r"], o["T"] = float(o["K"]), float(o["r"]), float(o["T"])
        for k in ("n_steps", "n_paths", "basis", "type", "seed", "rule"):
            o[k] = int(o[k])
    return AmericanPrice.apply(S0, sigma, fixed, amc_ctx, prec)
