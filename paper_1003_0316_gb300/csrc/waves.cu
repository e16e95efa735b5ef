// Memory-wave planner for the polarization of many q points whose projections do not fit in
// device memory together (the 64-q uneven mesh workload holds ~470 GB of projections): every q
// goes to one wave, and per wave the projections, the polarization workspace and the outputs
// must fit in a byte budget. First-fit decreasing: q points in order of decreasing footprint,
// each into the first wave with room (a new wave when none has). Host code only.
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
  const int64_t K0 = 0;
  const int nb0 = 1;
  // workspace that a launch needs once, whatever its q points (per-SM scratch)
  const size_t shared = pol_ws(1, &K0, &nb0, nw, precision);
  std::vector<size_t> foot(nq);
  for (int q = 0; q < nq; ++q) {
    const size_t ws = pol_ws(1, &K[q], &nb[q], nw, precision);
    foot[q] = size_t(K[q]) * size_t(nb[q]) * elem + (ws > shared ? ws - shared : 0) +
              size_t(nw) * size_t(nb[q]) * size_t(nb[q]) * 16 + 3 * 256;
    if (foot[q] + shared > budget)
      return set_error(GW_EINVAL, "q=%d alone needs %zu bytes, above the budget of %zu", q,
                       foot[q] + shared, budget);
  }
  std::vector<int> order(nq);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return foot[a] > foot[b]; });
  std::vector<size_t> used;
  for (int q : order) {
    int w = 0;
    while (w < int(used.size()) && used[w] + foot[q] > budget) ++w;
    if (w == int(used.size())) used.push_back(shared);
    used[w] += foot[q];
    wave_of_q[q] = w;
  }
  *nwaves = int(used.size());
  return GW_OK;
}

}  // namespace gw
