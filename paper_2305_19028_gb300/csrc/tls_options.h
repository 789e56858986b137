// Range checks of the numeric and switch fields of tls_options, shared by tls_factor and
// tls_batch_factor: every count bounded (so that no option turns a loop of the factor ladder or
// of PCGTLS into an unbounded one), every switch 0 or 1, every real finite and non-negative.
#pragma once

#include "../../include/tls.h"

#include <cmath>

namespace tls {

// nullptr when every field is in range, else what is wrong (tls_factor and tls_batch_factor
// add the rules that depend on the context: mode_A = 2 and factor = 1 on dense contexts only,
// mode_A = 1 in the packed batch)
inline const char* options_error(const tls_options& o) {
  if (o.u != TLS_FP32 && o.u != TLS_FP64) return "u must be FP32 or FP64";
  if (o.mode_A < 0 || o.mode_A > 2) return "mode_A must be 0, 1 or 2";
  if (o.factor < 0 || o.factor > 1) return "factor must be 0 or 1";
  auto flag = [](int v) { return v == 0 || v == 1; };
  auto count = [](int v, int lo, int hi) { return v >= lo && v <= hi; };
  auto real = [](double v) { return std::isfinite(v) && v >= 0.0; };
  if (!flag(o.cg_fixed) || !flag(o.psi_rule_ge) || !flag(o.gram_simt) || !flag(o.shift_first) ||
      !flag(o.fallback) || !flag(o.stall_fallback) || !flag(o.reproducible))
    return "cg_fixed, psi_rule_ge, gram_simt, shift_first, fallback, stall_fallback and "
           "reproducible must be 0 or 1";
  if (!count(o.cg_max, 1, 100000)) return "cg_max must be in [1, 100000]";
  if (!count(o.ls_iters, 0, 100000)) return "ls_iters must be in [0, 100000]";
  if (!count(o.max_shifts, 0, 30)) return "max_shifts must be in [0, 30]";
  if (!count(o.constraint_iters, 0, 100000)) return "constraint_iters must be in [0, 100000]";
  if (!real(o.cg_tol)) return "cg_tol must be finite and >= 0";
  if (std::isnan(o.psi_accept) || o.psi_accept < 0.0) return "psi_accept must be >= 0";
  if (!real(o.constr_guard)) return "constr_guard must be finite and >= 0";
  if (!real(o.stall_ratio)) return "stall_ratio must be finite and >= 0";
  if (!real(o.hybrid_ratio)) return "hybrid_ratio must be finite and >= 0";
  return nullptr;
}

}  // namespace tls
