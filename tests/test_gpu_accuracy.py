"""Accuracy of the precision forms, per D, against the float64 oracle (the
mixed-precision row: binary32 evaluation and products with float-float
interpolation; the float-float row: every value in float-float, the
products from the FMA two-product; compared with plain binary32 and
float64).

For each D and input family the GPU results in float32, mixed and float64
are compared with the oracle's float64 recurrence; the relative L-infinity
error max|z - z64| / max|z64| is printed (run with -s to see the table) and
checked against the forward-error bound (gamma_{3D+1}(u) + gamma_{3D+1}(u64))
* zabs, with u the working precision of the interpolation's inputs (2^-24:
the mixed form still rounds evaluations and products to binary32)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1608_00206_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U32, U64 = 2.0 ** -24, 2.0 ** -53


@pytest.fixture(scope="module")
def hc():
    from paper_1608_00206_gb300.build import build
    build()
    import paper_1608_00206_gb300 as hc
    return hc


def _run(hc, x, y, **kw):
    z = hc.convolve(torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV), **kw)
    return z.cpu().numpy().reshape(-1).astype(np.float64)


FAMILIES = {
    "pmf-exponential": lambda D, s: inputs.prob_exponential_pair(D, s),
    "uniform01": lambda D, s: tuple(v.astype(np.float64) for v in inputs.uniform01_pair(D, s)),
    "normal": lambda D, s: inputs.normal_pair(D, s, dtype=np.float64),
}


@pytest.mark.parametrize("family", sorted(FAMILIES))
def test_error_per_D_against_float64_oracle(hc, family):
    rows = []
    for D in (6, 8, 10, 12, 14, 16):
        x64, y64 = FAMILIES[family](D, 77 + D)
        x32, y32 = x64.astype(np.float32), y64.astype(np.float32)
        ref = oracle.convolve(x32.astype(np.float64), y32.astype(np.float64), threads=16)
        za = oracle.zabs(x32, y32)
        scale = np.abs(ref).max()
        errs = {}
        for name, kw, xs, ys in (("fp32", {}, x32, y32), ("mixed", {"mixed": True}, x32, y32),
                                 ("ff", {"mixed": "ff"}, x32, y32),
                                 ("fp64", {}, x32.astype(np.float64), y32.astype(np.float64))):
            z = _run(hc, xs, ys, **kw)
            err = np.abs(z - ref)
            if name == "ff":
                # float-float operations (u about 2^-47, bounded with 2^-44),
                # one binary32 rounding at the end, the float64 reference's own
                bound = ((oracle.gamma(3 * D + 1, 2.0 ** -44) + oracle.gamma(3 * D + 1, U64)) * za
                         + U32 * np.abs(ref))
            else:
                u = U64 if name == "fp64" else U32
                bound = (oracle.gamma(3 * D + 1, u) + oracle.gamma(3 * D + 1, U64)) * za
            assert np.all(err <= bound), (family, D, name)
            errs[name] = float(err.max() / scale)
        assert errs["fp64"] == 0.0  # bitwise equal to the oracle's own recurrence
        # float-float is within a few binary32 roundings of the scale, far
        # below the forms that round products to binary32
        assert errs["ff"] <= 4 * U32 and errs["ff"] <= errs["fp32"] / 10, (family, D)
        rows.append((D, errs["fp32"], errs["mixed"], errs["ff"]))
    print(f"\n{family}: D, rel. L-inf error vs float64 oracle (fp32, mixed, ff)")
    for D, e32, emx, eff in rows:
        print(f"  D={D:2d}  fp32 {e32:.3e}  mixed {emx:.3e}  ff {eff:.3e}  "
              f"fp32/ff {e32 / max(eff, 1e-300):.0f}")
