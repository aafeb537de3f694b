"""Score error of every form against the FP64 oracle as the background
covariance's condition number grows (224-band Gaussian cubes, GPU).

Prints the table; asserts each form's stated bar over the range of kappa on
which it is claimed: FP64 and FP64E (double-float score) 1e-9 up to 1e6; FP32
and 3xTF32 1e-4 up to 1e6 (the scatter's compensated FP32 sums keep them near
5e-5 there); TF32 5e-3 up to 1e4; BF16 4e-2 up to 1e4 (max relative delta error
over all pixels).  The cubes have the 224-band workload's width, 1024 px.  The
tensor-core forms take S2 on the tensor cores here (float lines: the TC
scatter route)."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import need_gpu, rel_err, run_gpu

pytestmark = pytest.mark.gpu

KAPPAS = [1e2, 1e3, 1e4, 1e5, 1e6]
BARS = {"fp64": (1e-9, 1e6), "fp64e": (1e-9, 1e6), "fp32": (1e-4, 1e6), "tf32x3": (1e-4, 1e6),
        "tf32": (5e-3, 1e4), "bf16": (4e-2, 1e4)}


@pytest.fixture(scope="module")
def table():
    need_gpu()
    out = {}
    for kappa in KAPPAS:
        cube = synth.gen_lines(synth.cov_c3(kappa, width=1024, bands=224, seed=2), 0, 4)
        ref = oracle.run_cube(cube, warmup=0)
        for form in BARS:
            got, _ = run_gpu(cube, form=form, warmup=0)
            out[(form, kappa)] = rel_err(got["delta"], ref["delta"])
    print("\nmax relative delta error, 4 lines x 1024 px x 224 bands")
    print("kappa   " + "".join(f"{f:>11s}" for f in BARS))
    for kappa in KAPPAS:
        print(f"{kappa:7.0e} " + "".join(f"{out[(f, kappa)]:11.2e}" for f in BARS))
    return out


@pytest.mark.parametrize("form", sorted(BARS))
def test_form_error_bar(table, form):
    bar, kmax = BARS[form]
    for kappa in KAPPAS:
        if kappa <= kmax:
            assert table[(form, kappa)] <= bar, (form, kappa, table[(form, kappa)])
