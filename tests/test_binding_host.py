"""Host logic of the Python binding (no GPU): the precision codes match the C
ABI's #defines in include/rqr.h, the status names match its RQR_ERR_* codes,
the precision a call gets from its dtype and prec= argument, the refusals
(unknown names or codes, data of the wrong type), and the leading dimension
passed for column-major views (padded, one row or column, empty)."""
import os
import re

import pytest
import torch

from paper_1505_08115_gb300 import rqr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _defines(prefix):
    text = open(os.path.join(ROOT, "include", "rqr.h")).read()
    return {k: int(v) for k, v in re.findall(r"#define (" + prefix + r"\w+) (-?\d+)", text)}


def test_precision_codes_match_the_header():
    d = _defines("RQR_")
    assert rqr.PRECISIONS == {"fp64": d["RQR_FP64"], "fp32": d["RQR_FP32"], "tf32": d["RQR_TF32"],
                              "3xbf16": d["RQR_3XBF16"], "3xtf32": d["RQR_3XTF32"], "fp64x": d["RQR_FP64X"]}
    assert (rqr.FP64, rqr.FP32, rqr.TF32, rqr.BF16X3, rqr.TF32X3, rqr.FP64X) == \
        (d["RQR_FP64"], d["RQR_FP32"], d["RQR_TF32"], d["RQR_3XBF16"], d["RQR_3XTF32"], d["RQR_FP64X"])
    assert (rqr.SKETCH_DOWNDATE, rqr.SKETCH_RESAMPLE) == (d["RQR_SKETCH_DOWNDATE"], d["RQR_SKETCH_RESAMPLE"])
    assert (rqr.BATCH_QRCP, rqr.BATCH_URV, rqr.BATCH_DESC_LEN) == \
        (d["RQR_BATCH_QRCP"], d["RQR_BATCH_URV"], d["RQR_BATCH_DESC_LEN"])


def test_status_names_cover_the_header_codes():
    errs = {v for k, v in _defines("RQR_").items() if k.startswith("RQR_ERR_") or k == "RQR_OK"}
    assert errs <= set(rqr.STATUS)


def test_precision_from_dtype_and_prec():
    f64, f32 = torch.float64, torch.float32
    assert rqr._prec(f64) == rqr.FP64 and rqr._prec(f64, emulated=True) == rqr.FP64X
    assert rqr._prec(f32) == rqr.FP32
    for name in ("fp64", "fp64x", "tf32", "3xbf16", "3xtf32"):
        assert rqr._prec(f64, prec=name) == rqr.PRECISIONS[name]
        assert rqr._prec(f64, prec=rqr.PRECISIONS[name]) == rqr.PRECISIONS[name]
    assert rqr._prec(f32, prec="fp32") == rqr.FP32
    # prec= wins over emulated=
    assert rqr._prec(f64, emulated=True, prec="fp64") == rqr.FP64


@pytest.mark.parametrize("dtype,prec", [(torch.float64, "bf16"), (torch.float64, 17), (torch.float64, "fp32"),
                                        (torch.float32, "tf32"), (torch.float32, "fp64x"), (torch.float16, None)])
def test_precision_refusals(dtype, prec):
    with pytest.raises(rqr.RQRError):
        rqr._prec(dtype, prec=prec)


def test_leading_dimension_of_column_major_views():
    assert rqr._ld(rqr.colmajor(torch.randn(5, 3))) == 5
    big = torch.zeros((3, 8), dtype=torch.float64).mT          # 8 x 3, ld 8
    assert rqr._ld(big[:5, :]) == 8                             # padded leading dimension
    assert rqr._ld(rqr.empty_colmajor(1, 4, device="cpu")) == 1
    assert rqr._ld(torch.randn(5, 1)) == 5                      # one column: either layout is column-major
    assert rqr._ld(rqr.empty_colmajor(0, 3, device="cpu")) == 1
    assert rqr._ld(rqr.empty_colmajor(6, 0, device="cpu")) == 6
    with pytest.raises(rqr.RQRError):
        rqr._ld(torch.randn(5, 3))                              # row-major
    with pytest.raises(rqr.RQRError):
        rqr._ld(torch.randn(3, 8)[:, ::2])                      # strided rows
