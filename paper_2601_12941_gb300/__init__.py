"""GB300-native local-subset 2D DIC (IC-GN, ZNSSD, cubic B-spline, frontier-wave
reliability-guided propagation) behind a C-ABI library, libdic.so, whose calls
this package re-exports under the same names."""
from .binding import (DIC_AFFINE, DIC_BF16, DIC_BICUBIC, DIC_BSPLINE3, DIC_F32, DIC_F64, DIC_FP64,  # noqa: F401
                      DIC_MIXED, DIC_QUADRATIC, DIC_RIGID, DIC_U16, DIC_U8, EXPORTS, N_PARAMS,
                      PT_FLAT, PT_LOW_ZNCC, PT_MAX_ITER, PT_NOT_IN_ROI, PT_NOT_REACHED, PT_OK,
                      PT_OUT_OF_BOUNDS, PT_SINGULAR, SHAPES, INTERPS, INITS, Correlation, DicError,
                      dic_correlate, dic_correlate_sequence, dic_create, dic_default_params, dic_destroy,
                      dic_get_coefficients, dic_get_params, dic_get_results, dic_get_timing,
                      dic_last_error, dic_set_deformed, dic_set_params, dic_set_reference,
                      load, make_image, params)
