// Internal device-side field handle of libfrpcpf (not part of the C ABI).
#pragma once
#include <utility>
#include <vector>

#include "internal.hpp"
#include "kdispatch.hpp"

// Recorded forward window for the adjoint (fr_adjoint_record).
struct AdjRecord {
  int active = 0;
  int n_steps = 0, ckpt_every = 0, n_ckpt = 0;
  int64_t step0 = 0;       // field step count at the start of the window
  char* ws = nullptr;      // caller workspace
  size_t bytes = 0;
  size_t off_ckpt = 0, off_stage = 0, off_times = 0, off_Y = 0, off_lamuo = 0, off_lamU = 0, off_Lp = 0,
         off_Lu = 0, off_Lk = 0, off_coefp = 0, off_cs = 0, off_lv = 0,
         off_trd = 0,   // mixed fields: FP64 shadow arrays (traces, state, stage input,
         off_u64 = 0, off_stg64 = 0, off_acc64 = 0, off_rp64 = 0, off_fc64 = 0, off_mc64 = 0,  // RK accumulator,
                        // partial divergence, common flux, metric records) of the FP64 recomputation
         off_pstage = 0, off_lpsi0 = 0;  // preconditioning: pseudo stage inputs, dR_p/dpsi0 adjoint
  int precond = 0, n_pseudo = 0;  // the window starts with the t = 0 preconditioning (n_pseudo iterations)
  int adj_blocks = 0;
};

struct fr_field {
  int dim = 0, etype = 0, order = 0, nu = 0, nf = 0, precision = 0;
  int64_t E = 0;
  frp::KArgs args{};
  frp::KernelSet ks{};
  fr_params prm{};
  int64_t nstep = 0;
  int64_t n_precond_done = 0;
  int sticky = FR_OK;
  int mass_grid = 1;
  double* xfer = nullptr;  // E*nu doubles, staging for get/set in the mixed path
  AdjRecord rec;
  frp::ElemPar* ep_region = nullptr;  // per-element parameters (used by batch fields)
  // CUDA graphs of the launch sequences (captured on a private stream on
  // first use, replayed on the caller's stream): kGraphSteps RK steps, one
  // RK step, one preconditioning
  int use_graphs = 1;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t g_steps = nullptr, g_step1 = nullptr, g_pre = nullptr;
  // optional per-launch CUDA-event timing: [class] -> (start, stop) pairs
  int profiling = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof[4];
};

namespace frp {
int field_run_step(fr_field* f, cudaStream_t s, bool allow_precondition);
int field_stage_and_traces(fr_field* f, cudaStream_t s);
// psi0 = psi = phi - 1/2 and the traces of psi: the start of a preconditioning
int field_precondition_begin(fr_field* f, cudaStream_t s);
}  // namespace frp
