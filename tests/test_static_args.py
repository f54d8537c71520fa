"""Argument checks of the binding's cvo_eval_gradient_static, on the CPU: a
wrong shape, dtype, layout or device is refused with ValueError before the
library is called, so no kernel can read past the end of a buffer."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1904_02266_gb300 as cvo  # noqa: E402


def _args(n=10, m=7, D=5):
    x = torch.zeros((n, 3), dtype=torch.float32)
    z = torch.zeros((m, 3), dtype=torch.float32)
    fx = torch.zeros((n, D), dtype=torch.float32)
    fz = torch.zeros((m, D), dtype=torch.float32)
    out = torch.zeros(8, dtype=torch.float64)
    return x, fx, z, fz, out


def _params(color_mode=cvo.CVO_COLOR_KERNEL, D=5):
    # the ctypes struct itself: the checks run before the library is loaded
    p = cvo.cvo_params()
    p.color_mode, p.feat_dim = color_mode, D
    return p


def _call(x, fx, z, fz, out, params=None):
    params = params or _params()
    cvo.cvo_eval_gradient_static(x, fx, z, fz, params, np.eye(4), 0.1, out)


@pytest.mark.parametrize("case", ["x_cols", "z_cols", "fx_rows", "fz_width", "x_f64", "fz_f64",
                                  "out_f32", "out_short", "x_noncontig", "cpu", "x_empty",
                                  "fx_missing"])
def test_bad_arguments_are_refused_before_any_launch(case):
    x, fx, z, fz, out = _args()
    if case == "x_cols":
        x = torch.zeros((10, 4), dtype=torch.float32)
    elif case == "z_cols":
        z = torch.zeros((7, 2), dtype=torch.float32)
    elif case == "fx_rows":
        fx = torch.zeros((9, 5), dtype=torch.float32)
    elif case == "fz_width":
        fz = torch.zeros((7, 3), dtype=torch.float32)
    elif case == "x_f64":
        x = x.double()
    elif case == "fz_f64":
        fz = fz.double()
    elif case == "out_f32":
        out = out.float()
    elif case == "out_short":
        out = torch.zeros(7, dtype=torch.float64)
    elif case == "x_noncontig":
        x = torch.zeros((3, 10), dtype=torch.float32).t()
    elif case == "x_empty":
        x = torch.zeros((0, 3), dtype=torch.float32)
    elif case == "fx_missing":
        fx = None
    # "cpu": well-formed tensors that are not on a GPU
    with pytest.raises(ValueError):
        _call(x, fx, z, fz, out)


def test_features_are_not_needed_without_a_label_product():
    x, _, z, _, out = _args()
    p = _params(cvo.CVO_COLOR_NONE)
    # only the device check is left to fail on a CPU tensor
    with pytest.raises(ValueError, match="CUDA"):
        _call(x, None, z, None, out, p)
