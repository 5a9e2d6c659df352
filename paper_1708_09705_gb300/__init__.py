"""GB300 hot path of Gaussian-process 3-D extinction mapping with EP
(Sale & Magorrian 2018): sparse sightline-integrated covariance assembly and
parallel expectation propagation with PCG-driven posterior marginals, in
hand-written CUDA for sm_103a behind the C ABI of include/gmead.h."""
from .gmead import (Config, Context, GmError, build_cov, config_from_catalogue,  # noqa: F401
                    default_config, ep_init, ep_sweep, get_posterior, lib, predict,
                    PREC_FP32, PREC_FP64, FORM_LINEAR, FORM_LOGNORMAL, TAPER_HARD,
                    TAPER_WENDLAND, LIK_GAUSS_IN_A, LIK_GAUSS_IN_LNA, EXPORTS, LIB_PATH,
                    COV_QUADRATURE, COV_SURROGATE, QUAD_GL, QUAD_BAND)
