// absorber.h -- the absorbing layers inside the pads (the layers [lambda, lambda, 6 lambda] of
// the Fig. 1 benchmark paragraph of arXiv 2506.15411; the paper does not give their profile).
//
// Inside a layer of L voxels, a voxel at depth t (1 on the innermost layer voxel, L on the
// outer face) gets k^2 = k_vac^2 (eps_r + i sigma) with
//     sigma = sigma_max (t / L)^p,
//     sigma_max = (p + 1) n_bg ln(1 / round_trip) / (k_vac L pitch),
// which makes a normally incident plane wave keep the amplitude round_trip after crossing the
// layer and back, in the weak-absorption estimate Im k = k_vac sigma / (2 n_bg).  Where layers
// of different axes overlap (edges, corners) their profiles add, or the largest one applies.
// Defaults: round_trip 1e-4, p = 2, profiles adding.  Shared by the plan's set-up (host) and
// the allocation-free splitting (device), so both compute the same sigma.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

#include "fft_radix.cuh"   // CBS_HD

namespace cbs {

constexpr double kLayerRoundTrip = 1e-4;
constexpr double kLayerPower = 2.0;

struct LayerSpec {
  double round_trip;   // in (0, 1)
  double power;        // ramp exponent p > 0
  int corner_max;      // 0: overlapping profiles add; 1: the largest applies
};

// The description's layer fields with their defaults (exactly 0 selects the default; other
// values out of range fail layer_spec_valid).
inline LayerSpec layer_spec(double round_trip, double power, int corner) {
  LayerSpec s;
  s.round_trip = round_trip == 0 ? kLayerRoundTrip : round_trip;
  s.power = power == 0 ? kLayerPower : power;
  s.corner_max = corner;
  return s;
}

inline bool layer_spec_valid(const LayerSpec& s) {
  return s.round_trip > 0 && s.round_trip < 1 && s.power > 0 && s.power <= 16 && (s.corner_max == 0 || s.corner_max == 1);
}

// sigma_max of a layer of L voxels (0 for L = 0).
CBS_HD double layer_sigma_max(const LayerSpec& s, double n_bg, double kvac, int L, double pitch) {
  return L > 0 ? (s.power + 1.0) * n_bg * log(1.0 / s.round_trip) / (kvac * L * pitch) : 0.0;
}

CBS_HD double layer_ramp(double t, double p) { return p == 2.0 ? t * t : pow(t, p); }

// sigma along one axis of n voxels with layers of lo and hi voxels (peak values slo, shi).
CBS_HD double layer_axis_sigma(int i, int n, int lo, int hi, double slo, double shi, double p) {
  if (i < lo) return slo * layer_ramp((double)(lo - i) / lo, p);
  if (i >= n - hi) return shi * layer_ramp((double)(i - (n - hi - 1)) / hi, p);
  return 0.0;
}

// sigma of a voxel from its three axis profiles.
CBS_HD double layer_combine(double sx, double sy, double sz, int corner_max) {
  return corner_max ? fmax(fmax(sx, sy), sz) : sx + sy + sz;
}

}  // namespace cbs
