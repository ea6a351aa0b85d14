"""The exponential step of the forward pass (Sec. 2.2.1: the stored S is
S0 exp(x)) on its own, through lsmc_exp: the double-precision exponential
(Tang's table-driven method for |x| < 512, CUDA's exp beyond) within one unit
in the last place of exp(x) computed in extended precision (numpy's long
double: binary128 on the Arm GPU hosts), over the whole double range in
which it is finite and across the switch at |x| = 512 (measured: 0.998 ulp
and 0.864 ulp); and the float-pair exponential within 2e-14 relative of the
same reference for |x| <= 70 (tests/test_exp_df.py emulates it on the CPU)."""
import numpy as np
import pytest

from gpu_common import torch_cuda
from paper_2206_03719_gb300 import lsmc as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = torch_cuda()
    from paper_2206_03719_gb300 import build
    build.build()
    return t


def _gpu_exp(torch, x, precision):
    if precision == L.LSMC_DF:
        hi = x.astype(np.float32)
        lo = (x - hi.astype(np.float64)).astype(np.float32)
        dx = torch.from_numpy(np.stack([hi, lo], axis=-1)).cuda()
        dy = torch.empty_like(dx)
    else:
        dx = torch.from_numpy(x).cuda()
        dy = torch.empty_like(dx)
    L.lsmc_exp(dx.data_ptr(), dy.data_ptr(), x.size, precision)
    torch.cuda.synchronize()
    y = dy.cpu().numpy()
    if precision == L.LSMC_DF:
        return y[..., 0].astype(np.longdouble) + y[..., 1].astype(np.longdouble)
    return y


def _ulp_err(y, x):
    ref = np.exp(x.astype(np.longdouble))
    ulp = np.spacing(np.abs(ref.astype(np.float64))).astype(np.longdouble)
    return np.abs(y.astype(np.longdouble) - ref) / ulp


def test_fp64_exponential_within_one_ulp(torch):
    if np.finfo(np.longdouble).nmant < 60:
        pytest.skip("no extended-precision long double on this host")
    rng = np.random.default_rng(7)
    x = np.concatenate([
        rng.uniform(-12.0, 12.0, 1 << 22),            # the range of the paths' log prices
        rng.uniform(-708.0, 709.0, 1 << 20),           # the whole finite range
        rng.uniform(-513.0, -511.0, 1 << 16), rng.uniform(511.0, 513.0, 1 << 16),
        np.array([0.0, 1e-300, -1e-300, 511.9999999, 512.0, -512.0, 512.0000001, 709.7,
                  -708.3, 1.0, -1.0, np.log(2.0), 0.5 * np.log(2.0) / 128.0]),
    ])
    y = _gpu_exp(torch, x, L.LSMC_FP64)
    err = _ulp_err(y, x)
    tang = np.abs(x) < 512.0
    print("exp_f64: worst %.3f ulp (Tang region), %.3f ulp (CUDA's exp beyond 512)"
          % (err[tang].max(), err[~tang].max()))
    assert err[tang].max() <= 1.0
    # CUDA documents its double exp within 1 ulp; the library relies on it there
    assert err[~tang].max() <= 1.0
    assert y[x == 0.0][0] == 1.0


def test_float_pair_exponential_close_to_exact(torch):
    if np.finfo(np.longdouble).nmant < 60:
        pytest.skip("no extended-precision long double on this host")
    rng = np.random.default_rng(8)
    # up to |x| = 70: beyond, the low part of exp(x) leaves float's normal
    # range (exp(-80) ~ 2e-35 has its low part among the subnormals, about
    # 4e-11 relative); the paths' exp(x) lies near 1
    x = np.concatenate([rng.uniform(-12.0, 12.0, 1 << 20), rng.uniform(-70.0, 70.0, 1 << 18),
                        np.array([0.0, 1e-30, -1e-30, 1.0, -1.0, 70.0, -70.0])])
    # the pairs hold x exactly only to about 48 bits: compare with exp of the
    # value they hold
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    held = hi.astype(np.longdouble) + lo.astype(np.longdouble)
    y = _gpu_exp(torch, x, L.LSMC_DF)
    rel = np.abs(y - np.exp(held)) / np.exp(held)
    print("exp_df: worst relative error %.3g" % rel.max())
    assert rel.max() <= 2e-14
