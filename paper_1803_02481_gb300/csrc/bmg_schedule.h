// Level schedule: the single-GPU reading of the coarse-grid redistribution
// of Section 2.2 / Algorithm 2.  Levels at or above the threshold run as
// full-grid kernel launches; levels below it run inside one persistent
// thread block (k_coarse_cycle) or one thread-block cluster
// (k_coarse_cycle_cluster), which removes every per-level launch.  The
// threshold and the number of blocks minimise a V-cycle time model in the
// form of Eq. (Vmodel) of Section 3: each operation costs a latency (kernel
// launch, or block or cluster barrier inside the persistent kernel) plus
// max(bytes / bandwidth, flops / rate).
#pragma once

#include "bmg_internal.h"

namespace bmg {

struct CostParams {
  double launch_us;      // per kernel launch on a captured/queued stream
  double sync_us;        // per __syncthreads phase inside the persistent kernel
  double gpu_gbs;        // full-GPU streaming bandwidth (GB/s)
  double gpu_gflops64;   // full-GPU FP64 FMA-based rate (GFLOP/s)
  double gpu_gflops32;
  double cta_gbs;        // one thread block, L2-resident data (GB/s)
  double cta_gflops64;   // one thread block (one SM) FP64 rate
  double cta_gflops32;
  double cluster_sync_us;  // per cluster-barrier phase of the cluster kernel
};

// Parameters in use (defaults, or measured by bmg_calibrate).
CostParams& cost_params();

// Predicted time (microseconds) of one V-cycle with the given threshold, the
// levels below it run by `ctas` blocks (1: one block, more: a cluster whose
// blocks each work at one SM's rates).
double predict_vcycle_us(const Hierarchy* h, int threshold, int ctas);

// argmin over thresholds 1..L (and, with the point smoother, over one block
// or the largest cluster the device supports) of predict_vcycle_us, within
// what h->opt fixes; fills h->predicted_us, sets h->threshold and
// h->coarse_ctas.
void choose_schedule(Hierarchy* h);

// Microbenchmarks of the cost-model parameters (bmg_calibrate).
int calibrate(cudaStream_t s, double* out);

}  // namespace bmg
