// tune.cu -- launch tuning table: lanes per ray for a (step count, map size).
//
// Default rule: at least 16 samples per lane when the map has enough rays to
// fill the GPU several times over; otherwise keep 32 lanes per ray for
// parallelism.  synax_set_lanes_per_ray() installs a measured table (the
// autotuner in paper_2410_01136_gb300/tune.py times the candidates and
// writes it) or forces one value.
#include <atomic>

#include "synax_internal.h"

namespace synax {

namespace {
// table[i] = lanes per ray for n_steps in [kStepEdges[i], kStepEdges[i + 1])
constexpr int kBins = 8;
constexpr int kStepEdges[kBins + 1] = {0, 64, 128, 256, 512, 1024, 2048, 4096, 1 << 30};
std::atomic<int> g_table[kBins] = {};
std::atomic<int> g_force{0};

int bin_of(int n_steps) {
    for (int i = 0; i < kBins; ++i)
        if (n_steps < kStepEdges[i + 1]) return i;
    return kBins - 1;
}
}  // namespace

int lanes_per_ray(int n_steps, long long n_pix) {
    const int forced = g_force.load(std::memory_order_relaxed);
    if (forced) return forced;
    const int t = g_table[bin_of(n_steps)].load(std::memory_order_relaxed);
    if (t) return t;
    // enough rays for >= 4 waves of 152 SMs x 32 resident warps at 8 lanes/ray?
    const long long rays_needed_8 = 4LL * 152 * 32 * 4;
    if (n_steps >= 128 && n_pix >= rays_needed_8) return 8;
    if (n_steps >= 64 && n_pix >= rays_needed_8 / 2) return 16;
    return 32;
}

}  // namespace synax

using namespace synax;

extern "C" int synax_set_lanes_per_ray(int n_steps_min, int lanes) {
    if (!(lanes == 0 || lanes == 8 || lanes == 16 || lanes == 32)) return SYNAX_EINVAL;
    if (n_steps_min < 0) {
        g_force.store(lanes, std::memory_order_relaxed);
        return SYNAX_OK;
    }
    g_table[bin_of(n_steps_min)].store(lanes, std::memory_order_relaxed);
    return SYNAX_OK;
}
