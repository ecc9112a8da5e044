// score_launch.cuh -- maps a runtime scoring configuration (lanes per candidate G, row
// pipelining) and a row width onto the compile-time kernel instantiation.
//
// For a row of nch 16-byte chunks and G lanes per candidate, every lane loads
// NCH = ceil(nch / G) chunks.  Instantiated: NCH in {1..6, 8, 10} without pipelining and
// NCH <= 5 with it; G in the store type's three group sizes plus 32 for wide rows.
#pragma once

#include "kernels.cuh"
#include "score_dev.cuh"

namespace glv {

// Group sizes offered per store type: the default G0 and its half and double.
template <int DT>
struct Groups {
  static constexpr int G0 = default_group<DT>();
  static constexpr int kLo = G0 > 1 ? G0 / 2 : 1;
  static constexpr int kHi = G0 * 2;
};

inline bool nch_supported(int n, bool pipe) {
  if (pipe) return n >= 1 && n <= 5;
  return (n >= 1 && n <= 6) || n == 8 || n == 10;
}

// Call f.template go<DT, G, NCH, PIPE>() for the requested configuration.
template <int DT, int G, class F>
cudaError_t dispatch_nch(int n, bool pipe, F& f) {
  if (pipe) {
    switch (n) {
      case 1: return f.template go<DT, G, 1, true>();
      case 2: return f.template go<DT, G, 2, true>();
      case 3: return f.template go<DT, G, 3, true>();
      case 4: return f.template go<DT, G, 4, true>();
      case 5: return f.template go<DT, G, 5, true>();
      default: return cudaErrorInvalidValue;
    }
  }
  switch (n) {
    case 1: return f.template go<DT, G, 1, false>();
    case 2: return f.template go<DT, G, 2, false>();
    case 3: return f.template go<DT, G, 3, false>();
    case 4: return f.template go<DT, G, 4, false>();
    case 5: return f.template go<DT, G, 5, false>();
    case 6: return f.template go<DT, G, 6, false>();
    case 8: return f.template go<DT, G, 8, false>();
    case 10: return f.template go<DT, G, 10, false>();
    default: return cudaErrorInvalidValue;
  }
}

// Smallest instantiated NCH >= n (extra slots are predicated off).
inline int round_nch(int n, bool pipe) {
  while (n <= 10 && !nch_supported(n, pipe)) ++n;
  return n;
}

template <int DT, class F>
cudaError_t dispatch_score(int G, int nch, bool pipe, F& f) {
  const int n = round_nch((nch + G - 1) / G, pipe);
  if (G == Groups<DT>::kLo) return dispatch_nch<DT, Groups<DT>::kLo>(n, pipe, f);
  if (G == Groups<DT>::G0) return dispatch_nch<DT, Groups<DT>::G0>(n, pipe, f);
  if (G == Groups<DT>::kHi) return dispatch_nch<DT, Groups<DT>::kHi>(n, pipe, f);
  if (G == 32) return dispatch_nch<DT, 32>(n, pipe, f);
  return cudaErrorInvalidValue;
}

// Effective configuration for a row of nch chunks: the tuned choice if it can serve the
// row, else the default group (or 32 lanes for wide rows) without pipelining.
struct ScoreConfig {
  int G;
  bool pipe;
};

template <int DT>
ScoreConfig effective_config(int nch, int tuned_G, bool tuned_pipe) {
  auto fits = [&](int G, bool pipe) { return G > 0 && round_nch((nch + G - 1) / G, pipe) <= 10; };
  if ((tuned_G == Groups<DT>::kLo || tuned_G == Groups<DT>::G0 || tuned_G == Groups<DT>::kHi || tuned_G == 32) &&
      fits(tuned_G, tuned_pipe))
    return {tuned_G, tuned_pipe};
  if (fits(Groups<DT>::G0, false)) return {Groups<DT>::G0, false};
  if (fits(Groups<DT>::kHi, false)) return {Groups<DT>::kHi, false};
  return {32, false};
}

}  // namespace glv
