// Cost model (host side): the loaded network and its FP64 host evaluation
// used by the DP-MLP planner.
#pragma once
#include <cstdint>

namespace qsa {
constexpr int kMlpIn = 37, kMlpH = 64;
constexpr int kMlpParams = kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;  // 6657

// x = [k/6, b_0..b_33 (physical target mask), N/34, log2(batch)/8]
void costmodel_features(int k, uint64_t phys_mask, int n, int batch, float* x);
bool costmodel_loaded();
// exp(f(x)) for the loaded network (seconds).
double costmodel_predict_seconds(int k, uint64_t phys_mask, int n, int batch);
}  // namespace qsa
