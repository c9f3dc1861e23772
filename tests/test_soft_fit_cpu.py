"""The soft score's weight calibration on the host (no GPU): the written-out
least-squares gradient and Adam update follow torch.optim.Adam on the same
standardised problem, given per-layer features (normally the CUDA forward's
mean sigmoids)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


class _Det:
    n = 16


class _Img:
    device = torch.device("cpu")


def test_fit_follows_torch_adam(monkeypatch):
    from paper_2108_12050_gb300 import soft
    rng = np.random.default_rng(4)
    N, n = 16, 16
    f = rng.uniform(0.0, 0.1, (N, n)) * rng.uniform(0.1, 3.0, n)   # uneven spreads
    y = rng.uniform(0.0, 8.0, N)
    monkeypatch.setattr(soft, "features", lambda det, imgs, tau, T=0.01: torch.tensor(f))
    tm = {}
    w, b, losses = soft.fit_weights(_Det(), [_Img()], y, tau=0.05, steps=200, timings=tm)
    assert set(tm) == {"features_s", "optimizer_s"}

    ft, yt = torch.tensor(f), torch.tensor(y)
    m, sd = ft.mean(0), ft.std(0) + 1e-6
    g = torch.Generator(device="cpu").manual_seed(0)
    v = (0.1 * torch.randn(n, generator=g, dtype=torch.float64)).requires_grad_(True)
    c = yt.mean().reshape(1).clone().requires_grad_(True)
    opt = torch.optim.Adam([v, c], lr=0.05)
    ref = []
    for _ in range(200):
        opt.zero_grad()
        loss = torch.mean((ft @ (v / sd) + (c - torch.dot(m / sd, v)) - yt) ** 2)
        loss.backward()
        opt.step()
        ref.append(float(loss.detach()))
    assert len(losses) == 200
    assert abs(losses[0] - ref[0]) < 1e-12
    assert abs(losses[-1] - ref[-1]) < 1e-6 * max(1.0, ref[0])
    with torch.no_grad():
        w_ref = (v / sd).float()
        b_ref = float(c - torch.dot(m / sd, v))
    assert torch.allclose(w, w_ref, rtol=1e-4, atol=1e-4)
    assert abs(float(b) - b_ref) < 1e-4 * max(1.0, abs(b_ref))
    # the returned (w, b) reproduce the fitted predictions
    pred = f @ w.double().numpy() + float(b)
    assert abs(np.mean((pred - y) ** 2) - losses[-1]) < 1e-3 * max(1.0, losses[0])
