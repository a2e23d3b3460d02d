// Lookups in the tuning table written by the autotuner (tuning.cu).
#pragma once

#include <string>

#include "common.cuh"

namespace fastpi {

struct CoreTiling;
// Tiling of the FP32 core SVD for an n x n core; false when the table has none.
bool tuned_core_tiling(int n, CoreTiling* out);
// Border rows / columns per append for a phase (0: Eq. 2, 1: Eq. 3) of target
// rank k_target in precision prec (0 FP64, 1 mixed); `fallback` when the table
// has no entry.
int64_t tuned_chunk(int prec, int phase, int64_t k_target, int64_t fallback);
// Register-tile class of a batched Jacobi problem whose longer side is dim
// (never below `natural`, the class its size needs).
int tuned_bucket_class(int prec, int dim, int natural);
// Smallest FP32 product (2 M N K flops) of the mixed form sent to the tensor
// cores; `fallback` when the table has none.
double tuned_tc_min_flops(double fallback);
// Replaces the table with the file at path (NULL: the built-in defaults);
// false, with the reason in *why, when the file cannot be read or parsed.
bool load_tuning(const char* path, std::string* why);
// Where the current table came from (a path, or "built-in defaults").
std::string tuning_source();

}  // namespace fastpi
