"""Device helpers the solvers rely on, checked against IEEE results computed on the host."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_recip_newton_within_ulps():
    """The FP64 pivot reciprocal of the path block solve (Newton-Raphson from the single-precision
    approximation) against the correctly rounded 1/x: within 2 ulp over magnitudes 1e-300..1e300,
    both signs, including the inputs outside float range that take the division."""
    from paper_2607_11340_gb300 import lib

    rng = np.random.default_rng(7)
    x = np.concatenate([10.0 ** rng.uniform(-300, 300, 20000), rng.uniform(0.5, 2.0, 20000),
                        10.0 ** rng.uniform(-12, 12, 20000), [1.0, 2.0, 3.0, 1e-37, 1e37, 1e-38, 1e38, 7e-300]])
    x = np.concatenate([x, -x])
    xd = torch.as_tensor(x, device="cuda")
    out = torch.empty_like(xd)
    lib.cr_device_check(lib.CR_CHECK_RECIP, xd, out)
    r = out.cpu().numpy()
    exact = 1.0 / x
    ulp = np.abs(r - exact) / np.spacing(np.abs(exact))
    assert ulp.max() <= 2.0, (ulp.max(), x[ulp.argmax()])


def test_fp64_sincos_within_ulps():
    """The FP64 sine and cosine of the kinematics against the host's: within 4 ulp of the result (the
    two sides' roundings together), near the zeros of sin and cos included, over |x| <= 1e4 and tiny
    arguments."""
    from paper_2607_11340_gb300 import lib

    rng = np.random.default_rng(11)
    x = np.concatenate([rng.uniform(-4, 4, 40000), rng.uniform(-1e4, 1e4, 20000), 10.0 ** rng.uniform(-300, 0, 5000),
                        np.arange(-20, 21) * (np.pi / 2), [1e-310]])
    xd = torch.as_tensor(x, device="cuda")
    for which, ref in ((lib.CR_CHECK_SIN, np.sin(x)), (lib.CR_CHECK_COS, np.cos(x))):
        out = torch.empty_like(xd)
        lib.cr_device_check(which, xd, out)
        r = out.cpu().numpy()
        ulp = np.abs(r - ref) / np.spacing(np.maximum(np.abs(ref), 1e-300))
        assert ulp.max() <= 4.0, (which, ulp.max(), x[ulp.argmax()])

