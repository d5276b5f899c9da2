"""The FP64 conductivity laws on the GPU (fem_law_eval), through the C ABI.

The FP64 element kernels evaluate k(u_q) and k'(u_q) with this device code
(the S of Algorithm 2, Section 4.2; k' for the tangent, Section 5.2).  The
sine law uses the library's own table-driven sin/cos; it is checked against
CUDA's sin/cos (torch on the GPU) and against the host's libm (numpy): at
most 2 units in the last place from libm (3 from CUDA's, itself within 2),
or 1e-21 absolute near a zero of the
function, over arguments spread across many periods, near multiples of
pi/128 (table points), near multiples of pi (zeros of sin), tiny values and
large values past the table reduction's range (which fall back to CUDA's
sincos).  Polynomial and piecewise-linear laws are checked against their
definitions in the oracle.
"""
import numpy as np
import pytest

import oracle as orc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2204_03893_gb300 as F  # noqa: E402


def _eval(kind, params, u):
    du = torch.tensor(u, dtype=torch.float64, device="cuda")
    k = torch.empty_like(du)
    dk = torch.empty_like(du)
    F.fem_law_eval(F.coeff(kind, params), du, du.numel(), k, dk)
    torch.cuda.synchronize()
    return du, k, dk


def _ulp_ok(got, ref, ulps=2.0, floor=1e-21):
    got, ref = np.asarray(got), np.asarray(ref)
    err = np.abs(got - ref)
    bound = ulps * np.spacing(np.abs(ref)) + floor
    return err <= bound, err / bound


def _arguments():
    rng = np.random.default_rng(7)
    parts = [rng.uniform(-40.0, 40.0, 200000),
             rng.uniform(0.0, 3.0, 50000),                          # 3u for u in [0, 1]
             np.arange(-4000, 4000) * (np.pi / 128) + rng.uniform(-1e-9, 1e-9, 8000),   # table points
             np.arange(-300, 300) * np.pi,                          # zeros of sin
             np.arange(-300, 300) * np.pi + np.pi / 2,              # zeros of cos
             rng.uniform(-1e-6, 1e-6, 1000), np.array([0.0, -0.0, 1e-300, 5e-324]),
             rng.uniform(2.5e4, 1e6, 2000) * rng.choice([-1, 1], 2000)]   # past the reduction's range
    return np.concatenate(parts)


def test_sine_law_matches_cuda_and_libm():
    x = _arguments()
    du, k, dk = _eval("sin", (0.0, 1.0, 1.0), x)      # k = sin(u), k' = cos(u)
    g_s, g_c = k.cpu().numpy(), dk.cpu().numpy()
    # libm is within 1 ulp of the exact value; CUDA's sin/cos within 2, so 3 against CUDA
    for ref_s, ref_c, what, ulps in ((np.sin(x), np.cos(x), "libm", 2.0),
                                     (torch.sin(du).cpu().numpy(), torch.cos(du).cpu().numpy(), "cuda", 3.0)):
        ok_s, r_s = _ulp_ok(g_s, ref_s, ulps)
        ok_c, r_c = _ulp_ok(g_c, ref_c, ulps)
        assert ok_s.all(), (what, "sin", x[~ok_s][:5], r_s.max())
        assert ok_c.all(), (what, "cos", x[~ok_c][:5], r_c.max())


def test_sine_law_parameters():
    u = np.random.default_rng(8).uniform(0.0, 1.0, 10000)
    _, k, dk = _eval("sin", (2.0, 1.0, 3.0), u)             # the 3D workloads' k = 2 + sin(3u)
    ok, _ = _ulp_ok(k.cpu().numpy(), 2.0 + np.sin(3.0 * u), ulps=3)
    assert ok.all()
    ok, _ = _ulp_ok(dk.cpu().numpy(), 3.0 * np.cos(3.0 * u), ulps=3)
    assert ok.all()


@pytest.mark.parametrize("law", [("poly", (1.0,)), ("poly", (1.0, 0.5, 0.25)), ("poly", (1.0, 0.0, 1.0)),
                                 ("poly", (0.3, -1.2, 0.7, 2.0, -0.1, 0.05, 0.01, -0.02)),
                                 ("pwlin", (0.0, 0.3, 0.6, 1.0, 1.0, 2.0, 1.5, 3.0))])
def test_polynomial_and_piecewise_laws(law):
    kind, params = law
    u = np.concatenate([np.random.default_rng(9).uniform(-0.5, 1.5, 5000), [0.0, 0.3, 0.6, 1.0]])
    _, k, dk = _eval(kind, params, u)
    ref = np.array([orc.kfun(kind, params, x) for x in u])
    scale = 1.0 + np.abs(ref)
    assert (np.abs(k.cpu().numpy() - ref[:, 0]) <= 1e-14 * scale[:, 0]).all()
    assert (np.abs(dk.cpu().numpy() - ref[:, 1]) <= 1e-13 * scale[:, 1]).all()


def test_law_eval_refuses_host_pointers():
    u = np.zeros(10)
    with pytest.raises(F.FemError) as ei:
        F.fem_law_eval(F.coeff("poly", (1.0,)), u, 10, u, u)
    assert ei.value.code == F.FEM_EINVAL


def test_fp32_law_code():
    """fem_law_eval_fp32: the FP32 law code of the FP32 and tensor-core
    element kernels.  Its sin/cos (CUDA's sincosf) against the sine and
    cosine of the same FP32 argument in FP64 (numpy): at most 3 FP32 units in
    the last place over |x| < 100 (multiples of pi/128 and of pi, tiny and
    spread arguments), 8 beyond; a polynomial law against its Horner form in
    FP32."""
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.uniform(-99.0, 99.0, 200000), rng.uniform(0.0, 3.0, 50000),
                        np.arange(-4000, 4000) * (np.pi / 128), np.arange(-30, 31) * np.pi,
                        np.arange(-30, 30) * np.pi + np.pi / 2, rng.uniform(-1e-6, 1e-6, 1000),
                        rng.uniform(100.0, 2e4, 2000) * rng.choice([-1, 1], 2000)]).astype(np.float32)
    du = torch.tensor(x.astype(np.float64), device="cuda")
    k = torch.empty(x.size, dtype=torch.float32, device="cuda")
    dk = torch.empty_like(k)
    F.fem_law_eval_fp32(F.coeff("sin", (0.0, 1.0, 1.0)), du, x.size, k, dk)
    torch.cuda.synchronize()
    xs = x.astype(np.float64)
    for got, ref in ((k.cpu().numpy(), np.sin(xs)), (dk.cpu().numpy(), np.cos(xs))):
        ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
        err = np.abs(got.astype(np.float64) - ref) / ulp
        inner = np.abs(xs) < 100.0
        assert err[inner].max() <= 3.0, err[inner].max()
        assert err[~inner].max() <= 8.0, err[~inner].max()
    # a quadratic law: the 3-term Horner of the FP32 kernels
    u = rng.uniform(-2.0, 2.0, 10000)
    du = torch.tensor(u, device="cuda")
    k = torch.empty(u.size, dtype=torch.float32, device="cuda")
    dk = torch.empty_like(k)
    F.fem_law_eval_fp32(F.coeff("poly", (1.0, 0.5, 0.25)), du, u.size, k, dk)
    torch.cuda.synchronize()
    uf = u.astype(np.float32).astype(np.float64)
    assert np.abs(k.cpu().numpy() - (1.0 + 0.5 * uf + 0.25 * uf ** 2)).max() <= 4e-7 * 3
    assert np.abs(dk.cpu().numpy() - (0.5 + 0.5 * uf)).max() <= 4e-7 * 3
    with pytest.raises(F.FemError):
        F.fem_law_eval_fp32(F.coeff("sin", (0.0, 1.0, 1.0)), np.zeros(4), 4, k, dk)
