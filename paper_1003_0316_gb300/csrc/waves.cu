// Memory-wave planner for the polarization of many q points whose projections do not fit in
// device memory together (the 64-q uneven mesh workload holds ~470 GB of projections): every q
// goes to one wave, and per wave the projections, the polarization workspace and the outputs
// must fit in a byte budget. First-fit decreasing: q points in order of decreasing footprint,
// each into the first wave with room (a new wave when none has); a wave's bytes are evaluated
// for its whole q list, since the workspace of one call is not a sum over its q. Host code
// only.
#include <algorithm>
#include <numeric>
#include <vector>

#include "gw_internal.cuh"

namespace gw {

static size_t pol_ws(int nq, const int64_t* K, const int* nb, int nw, int precision) {
  return precision == GW_FP64 ? pol_fp64_workspace(nq, K, nb, nw, PolOpts{})
                              : pol_tc_workspace(nq, K, nb, nw, precision, PolOpts{});
}

int plan_waves(int nq, const int64_t* K, const int* nb, int nw, int precision, size_t budget,
               int* wave_of_q, int* nwaves) {
  const size_t elem = precision == GW_FP64 ? 16 : 8;
  // projections and outputs of one q (plus the alignment of their allocations)
  std::vector<size_t> data(nq);
  for (int q = 0; q < nq; ++q)
    data[q] = size_t(K[q]) * size_t(nb[q]) * elem + size_t(nw) * size_t(nb[q]) * size_t(nb[q]) * 16 +
              3 * 256;
  // the bytes of a wave: its data and the workspace of one call over its q in increasing order
  // (the workspace is not additive over q: groups, and two slots when there are several)
  auto cost = [&](const std::vector<int>& qs) {
    std::vector<int64_t> Kw;
    std::vector<int> nbw;
    size_t b = 0;
    for (int q : qs) {
      Kw.push_back(K[q]);
      nbw.push_back(nb[q]);
      b += data[q];
    }
    return b + pol_ws(int(qs.size()), Kw.data(), nbw.data(), nw, precision);
  };
  std::vector<size_t> foot(nq);
  for (int q = 0; q < nq; ++q) {
    foot[q] = cost({q});
    if (foot[q] > budget)
      return set_error(GW_EINVAL, "q=%d alone needs %zu bytes, above the budget of %zu", q,
                       foot[q], budget);
  }
  std::vector<int> order(nq);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return foot[a] > foot[b]; });
  std::vector<std::vector<int>> waves;
  for (int q : order) {
    size_t w = 0;
    for (; w < waves.size(); ++w) {
      std::vector<int> t = waves[w];
      t.insert(std::upper_bound(t.begin(), t.end(), q), q);
      if (cost(t) <= budget) {
        waves[w] = t;
        break;
      }
    }
    if (w == waves.size()) waves.push_back({q});
    wave_of_q[q] = int(w);
  }
  *nwaves = int(waves.size());
  return GW_OK;
}

}  // namespace gw
