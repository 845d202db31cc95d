// Cost model (host side): the installed network and its FP64 host
// evaluation used by the DP-MLP planner.
#pragma once
#include <cstdint>
#include <memory>
#include <string>
#include <vector>

namespace qsa {
constexpr int kMlpIn = 37, kMlpH = 64;
constexpr int kMlpParams = kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;  // 6657

// A network's parameters (W1 b1 W2 b2 W3 b3), shared read-only by the
// process-wide slot, states it is attached to and planners using it.
using CostParams = std::vector<double>;
using CostModel = std::shared_ptr<const CostParams>;

// x = [k/6, b_0..b_33 (physical target mask), N/34, log2(batch)/8]
void costmodel_features(int k, uint64_t phys_mask, int n, int batch, float* x);
// The process-wide model (null if none is installed).
CostModel costmodel_global();
bool costmodel_loaded();
// exp(f(x)) in seconds for the given network.
double costmodel_eval(const CostParams& P, int k, uint64_t phys_mask, int n, int batch);
// exp(f(x)) for the process-wide network (NaN if none).
double costmodel_predict_seconds(int k, uint64_t phys_mask, int n, int batch);
}  // namespace qsa
