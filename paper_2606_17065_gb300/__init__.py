"""PIVOT on GB300: batched Black-76 implied volatility in LBR form with its
implicit-function-theorem adjoint and low-vega gating, as hand-written
sm_103a CUDA behind a small C ABI (include/pivot.h).

Importing the package does not load the CUDA library; the first call does,
and fails loudly if it has not been built.
"""
from .api import (GATES, MODES, ROW_ABOVE_UPPER, ROW_AT_INTRINSIC, ROW_AT_UPPER, ROW_BAD_INPUT,
                  ROW_BELOW_INTRINSIC, ROW_OK, BlackPrice, ImpliedVol, black_price, black_price_autograd,
                  black_price_backward, implied_volatility_autograd, iv, iv_backward, iv_forward_backward,
                  iv_guess, MlpTrainer, ImpliedVolBS, bs_implied_volatility_autograd, bs_iv, bs_iv_backward,
                  bs_iv_forward_backward, bs_price, new_counters, release_host_buffers)

__all__ = ["new_counters", "release_host_buffers", "bs_price", "bs_iv", "bs_iv_backward", "bs_iv_forward_backward", "ImpliedVolBS",
           "bs_implied_volatility_autograd", "iv_guess", "MlpTrainer", "black_price", "black_price_backward", "BlackPrice", "black_price_autograd", "iv", "iv_backward", "iv_forward_backward", "ImpliedVol", "implied_volatility_autograd",
           "GATES", "MODES", "ROW_OK", "ROW_BELOW_INTRINSIC", "ROW_ABOVE_UPPER", "ROW_BAD_INPUT", "ROW_AT_INTRINSIC",
           "ROW_AT_UPPER"]
