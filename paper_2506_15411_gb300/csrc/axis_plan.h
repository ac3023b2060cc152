// axis_plan.h -- host-side planning of one FFT axis for the in-place stages of fft_ip.cuh:
// the radices, their order, and the device tables (stages, twiddles, wave numbers).
//
// Used by the library (api.cu) and, compiled for the CPU, by the tests that run the stage
// code on the host.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <vector>

namespace cbs {

constexpr int kMaxAxisStages = 8;

// How the passes of this axis touch shared memory, for the bank-conflict model.
enum class AxisLayout {
  Rows,      // x passes: elements of a row contiguous; lanes take consecutive butterflies
  Cols,      // y pass: NCOL-column tiles, lanes take column pairs, then butterflies
  ColsZ      // z pass: as Cols, but the last DIF stage moves single columns (the fused
             // k-space stage), lanes taking columns, then butterflies
};

// Factor n into radices of {16, 13, 12, 11, 10, 9, 8, 7, 6, 5, 4, 3, 2} (at most max_radix):
// fewest stages, then the largest smallest radix (fewest threads per transform).  Returns
// false if n has another prime factor.  n = 1 gives the single radix 1.
inline bool factor_radices(int n, int max_radix, std::vector<int>& out) {
  static const int cand[] = {16, 13, 12, 11, 10, 9, 8, 7, 6, 5, 4, 3, 2};
  out.clear();
  if (n == 1) {
    out.push_back(1);
    return true;
  }
  std::vector<int> cur, best;
  auto better = [&](const std::vector<int>& a, const std::vector<int>& b) {
    if (b.empty()) return true;
    if (a.size() != b.size()) return a.size() < b.size();
    return *std::min_element(a.begin(), a.end()) > *std::min_element(b.begin(), b.end());
  };
  std::function<void(int, int)> dfs = [&](int rem, int maxr) {
    if (rem == 1) {
      if (better(cur, best)) best = cur;
      return;
    }
    if ((int)cur.size() >= kMaxAxisStages) return;
    for (int r : cand) {
      if (r > maxr || r > max_radix || rem % r) continue;
      cur.push_back(r);
      dfs(rem / r, r);
      cur.pop_back();
    }
  };
  dfs(n, 1 << 30);
  if (best.empty()) return false;
  out = best;   // largest first
  return true;
}

// Shared-memory wavefronts of one warp-wide access: lane l touches `width` bytes at byte
// address addr[l] (active[l]).  32 banks of 4 bytes; 8-byte accesses are served in two
// phases of 16 lanes, 16-byte ones in four of 8; within a phase the count is the largest
// number of distinct 4-byte words falling in one bank.
inline int warp_wavefronts(const long long* addr, const bool* active, int width) {
  const int per = width >= 16 ? 8 : (width == 8 ? 16 : 32);
  int total = 0;
  for (int ph = 0; ph < 32; ph += per) {
    std::vector<std::vector<long long>> bank(32);
    bool any = false;
    for (int l = ph; l < ph + per; ++l) {
      if (!active[l]) continue;
      any = true;
      for (int w = 0; w < width / 4; ++w) {
        const long long word = addr[l] / 4 + w;
        auto& b = bank[word % 32];
        if (std::find(b.begin(), b.end(), word) == b.end()) b.push_back(word);
      }
    }
    if (!any) continue;
    size_t mx = 0;
    for (auto& b : bank) mx = std::max(mx, b.size());
    total += (int)mx;
  }
  return total;
}

// Modelled shared-memory wavefronts of the element loads of one warp (items 0..31) over all
// stages of `order` (twiddle loads are conflict-free by the table layout), for a tile with
// ncol columns (column layouts) or rows of stride ld (row layout).
inline long long layout_cost(const std::vector<int>& order, int n, AxisLayout lay, int ncol) {
  long long cost = 0;
  int prod = 1;
  const int s = (int)order.size();
  for (int q = 0; q < s; ++q) {
    const int R = order[q];
    prod *= R;
    const int m = n / prod, L = R * m, nb = n / R;
    long long addr[32];
    bool act[32];
    const bool last = (q == s - 1);
    for (int r = 0; r < R; ++r) {
      int width = 8;
      for (int l = 0; l < 32; ++l) {
        act[l] = true;
        if (lay == AxisLayout::Rows) {
          const int t = l % nb;   // items beyond one row wrap to the next row (same banks)
          const int b = t / m, j = t % m;
          if (last && R % 2 == 0) {
            if (r >= R / 2) { act[l] = false; addr[l] = 0; continue; }
            width = 16;
            addr[l] = (long long)(b * L + j) * 8 + 16LL * r;
          } else {
            addr[l] = (long long)(b * L + j + r * m) * 8;
          }
        } else if (lay == AxisLayout::ColsZ && last) {
          const int col = l % ncol, t = (l / ncol) % nb;
          const int b = t / m, j = t % m;
          addr[l] = (long long)((b * L + j + r * m) * ncol + col) * 8;
        } else {
          width = 16;
          const int np = ncol / 2;
          const int p = l % np, t = (l / np) % nb;
          const int b = t / m, j = t % m;
          addr[l] = (long long)((b * L + j + r * m) * np + p) * 16;
        }
      }
      cost += warp_wavefronts(addr, act, width);
    }
  }
  return cost;
}

// The order of the radices for a layout: the permutation with the fewest modelled
// wavefronts; ties keep the largest-first order.
inline std::vector<int> order_radices(const std::vector<int>& radices, int n, AxisLayout lay, int ncol) {
  std::vector<int> perm = radices;
  std::sort(perm.begin(), perm.end());
  std::vector<int> best = radices;
  long long best_cost = layout_cost(radices, n, lay, ncol);
  do {
    const long long c = layout_cost(perm, n, lay, ncol);
    if (c < best_cost) {
      best_cost = c;
      best = perm;
    }
  } while (std::next_permutation(perm.begin(), perm.end()));
  return best;
}

// Modelled work of the stages of one z tile for a radix order: per stage, the rounds a warp
// group of nth threads makes over the stage's items, times the values an item holds.  The
// stages before the last take column pairs of each of the three components (and run twice:
// forward and inverse); the last, fused stage takes single columns with all three
// components and runs its forward and inverse butterflies in one item.  A stage whose items
// leave most threads idle in its last round costs a whole round.
inline long long z_balance_cost(const std::vector<int>& order, int n, int ncol, int nth) {
  long long cost = 0;
  const int s = (int)order.size();
  for (int q = 0; q < s; ++q) {
    const int R = order[q];
    if (q < s - 1) {
      const long long items = 3LL * (ncol / 2) * (n / R);
      cost += 2 * ((items + nth - 1) / nth) * 2 * R;
    } else {
      const long long items = (long long)ncol * (n / R);
      cost += ((items + nth - 1) / nth) * 6 * R;
    }
  }
  return cost;
}

// The order of the z axis' radices: the least modelled work (z_balance_cost), then the fewest
// modelled shared-memory wavefronts (layout_cost), then the largest-first order.
inline std::vector<int> order_radices_z(const std::vector<int>& radices, int n, int ncol, int nth) {
  std::vector<int> perm = radices;
  std::sort(perm.begin(), perm.end());
  std::vector<int> best = radices;
  long long bw = z_balance_cost(radices, n, ncol, nth), bc = layout_cost(radices, n, AxisLayout::ColsZ, ncol);
  do {
    const long long w = z_balance_cost(perm, n, ncol, nth);
    const long long c = layout_cost(perm, n, AxisLayout::ColsZ, ncol);
    if (w < bw || (w == bw && c < bc)) {
      bw = w;
      bc = c;
      best = perm;
    }
  } while (std::next_permutation(perm.begin(), perm.end()));
  return best;
}

// Device tables of an axis for a given radix order (see fft_ip.cuh): the stage table
// (2 int4 per stage), the twiddle table (complex64, w_n^{j k P_q} at tw_off_q + (k-1) m_q + j,
// computed in FP64 and rounded), and the wave numbers (p, q) of each position (scaled by the
// pitch: p = 2 pi fftfreq(k, n), q = p but 0 at the Nyquist frequency of an even n).
inline void axis_tables(int n, const std::vector<int>& order, std::vector<int4>& st, std::vector<float2>& tw,
                        std::vector<float2>& pq) {
  const double two_pi = 6.283185307179586476925287;
  auto bits = [](float f) {
    int i;
    std::memcpy(&i, &f, sizeof(i));
    return i;
  };
  const int s = (int)order.size();
  st.assign(2 * s, make_int4(1, 1, 1, 0));
  tw.clear();
  int prod = 1;
  for (int q = 0; q < s; ++q) {
    const int R = order[q];
    const int P = prod;   // n / L_q
    prod *= R;
    const int m = n / prod, L = R * m;
    st[2 * q] = make_int4(R, m, L, (int)tw.size());
    st[2 * q + 1] = make_int4(bits(1.0f / (float)m), bits(1.0f / (float)(n / R)), n / R, 0);
    if (q < s - 1)
      for (int k = 1; k < R; ++k)
        for (int j = 0; j < m; ++j) {
          const double a = -two_pi * (double)((long long)j * k * P % n) / (double)n;
          tw.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
        }
  }
  // position of frequency k: its mixed-radix digits d_q (d_0 least significant, base R_0)
  // weighted by m_q
  pq.assign(n, make_float2(0.f, 0.f));
  for (int k = 0; k < n; ++k) {
    int rem = k, pos = 0, pr = 1;
    for (int q = 0; q < s; ++q) {
      const int R = order[q];
      pr *= R;
      const int d = rem % R;
      rem /= R;
      pos += d * (n / pr);
    }
    const int f = (2 * k < n) ? k : k - n;
    const float p = (float)(two_pi * (double)f / (double)n);
    pq[pos] = make_float2(p, (2 * k == n) ? 0.f : p);
  }
}

}  // namespace cbs
