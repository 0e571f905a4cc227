// Hand-written discrete adjoint of the FR-PCPF march (C ABI:
// fr_adjoint_workspace_bytes, fr_adjoint_record, fr_adjoint_step).
//
// fr_adjoint_record runs the forward march from the current state and keeps
// the solution every ckpt_every steps in the caller's workspace.
// fr_adjoint_step sweeps backwards: per checkpoint segment it recomputes the
// forward steps, keeping the four RK stage inputs of each step, then applies
// the transpose of each RK4 step,
//   lam_k4 = dt/6 lam'          a4 = (dR/du)^T(U4) lam_k4
//   lam_k3 = dt/3 lam' + dt a4  a3 = (dR/du)^T(U3) lam_k3
//   lam_k2 = dt/3 lam' + dt/2 a3, a2 ...   lam_k1 = dt/6 lam' + dt/2 a2, a1 ...
//   lam = lam' + a4 + a3 + a2 + a1,
// with the vector-Jacobian products of kadj.cuh, and accumulates the
// gradient with respect to the stream-function coefficients.
#include <cmath>
#include <cstring>
#include <vector>

#include "field.cuh"
#include "kadj.cuh"

using namespace frp;

namespace {

#define CK(x)                                \
  do {                                       \
    if ((x) != cudaSuccess) return FR_ECUDA; \
  } while (0)

size_t al(size_t x) { return (x + 255) / 256 * 256; }

typedef void (*AdjFn)(const AdjArgs&, cudaStream_t);
typedef void (*TabFn)(const KArgs&, double*, cudaStream_t);
struct AdjSet {
  AdjFn a = nullptr, b = nullptr, c = nullptr;
  TabFn tab = nullptr;  // cos/sin table of the stream-function modes at the points
  int et = 1;
};

template <int DIM, int N>
void la(const AdjArgs& B, cudaStream_t s) {
  using LY = AdjLayout<DIM, N>;
  adj_a<DIM, N><<<(unsigned)((B.K.E + LY::ET - 1) / LY::ET), LY::THREADS, 0, s>>>(B);
}
template <int DIM, int N>
void lb(const AdjArgs& B, cudaStream_t s) {
  using LY = AdjLayout<DIM, N>;
  static bool init = false;
  if (!init) {
    cudaFuncSetAttribute(adj_b<DIM, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LY::SMEM);
    init = true;
  }
  adj_b<DIM, N><<<(unsigned)((B.K.E + LY::ET - 1) / LY::ET), LY::THREADS, LY::SMEM, s>>>(B);
}
template <int DIM, int N>
void lc(const AdjArgs& B, cudaStream_t s) {
  using LY = AdjLayout<DIM, N>;
  adj_c<DIM, N><<<(unsigned)((B.K.E + LY::ET - 1) / LY::ET), LY::THREADS, 0, s>>>(B);
}
template <int DIM, int N>
void ltab(const KArgs& A, double* cs, cudaStream_t s) {
  const int64_t n = A.E * (TS<DIM, N>::NU + TS<DIM, N>::NF);
  const int64_t g = (n + 255) / 256;
  k_coef_table<DIM, N><<<(unsigned)(g < 152 * 16 ? g : 152 * 16), 256, 0, s>>>(A, cs);
}
template <int DIM, int N>
AdjSet make_set() {
  AdjSet a;
  a.a = la<DIM, N>;
  a.b = lb<DIM, N>;
  a.c = lc<DIM, N>;
  a.tab = ltab<DIM, N>;
  a.et = AdjLayout<DIM, N>::ET;
  return a;
}

bool adj_kernels(const fr_field* f, AdjSet* out) {
  if (f->precision != FR_FP64) return false;
  if (f->etype == FR_QUAD) {
    switch (f->order) {
      case 1: *out = make_set<2, 2>(); return true;
      case 2: *out = make_set<2, 3>(); return true;
      case 3: *out = make_set<2, 4>(); return true;
      case 4: *out = make_set<2, 5>(); return true;
      case 5: *out = make_set<2, 6>(); return true;
      case 6: *out = make_set<2, 7>(); return true;
    }
  }
  if (f->etype == FR_HEX) {
    switch (f->order) {
      case 1: *out = make_set<3, 2>(); return true;
      case 2: *out = make_set<3, 3>(); return true;
      case 3: *out = make_set<3, 4>(); return true;
    }
  }
  return false;
}

__global__ void k_pack_lam(double* L, const double* dphi, const double* dpsi, int64_t E, int NU) {
  const int64_t n = E * NU;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / NU, i = g % NU;
    L[(e * 2 + 0) * NU + i] = dphi[g];
    L[(e * 2 + 1) * NU + i] = dpsi ? dpsi[g] : 0.0;
  }
}

__global__ void k_unpack_lam(const double* L, double* out, int64_t E, int NU) {
  const int64_t n = E * NU;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / NU, i = g % NU;
    out[g] = L[(e * 2 + 0) * NU + i];
    out[n + g] = L[(e * 2 + 1) * NU + i];
  }
}

// out[m] = sum over blocks of coefp[b][m], in block order
__global__ void k_coef_reduce(const double* coefp, int nblocks, int M2, double* out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M2) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += coefp[(int64_t)b * M2 + m];
  out[m] = s;
}

struct Sizes {
  size_t ckpt_slot, stage_slot, total;
  int n_ckpt;
};

Sizes sizes(const fr_field* f, int n_steps, int ck, int adj_blocks) {
  Sizes z;
  const size_t ndof = (size_t)f->E * f->nu;
  z.n_ckpt = (n_steps + ck - 1) / ck;
  z.ckpt_slot = al(2 * ndof * 8 + 8);
  z.stage_slot = al(2 * ndof * 8);
  const size_t nf2 = (size_t)f->E * 2 * f->nf * 8;
  size_t t = 0;
  t += (z.n_ckpt + 1) * z.ckpt_slot;
  t += (size_t)ck * 4 * z.stage_slot;
  t += al((size_t)ck * 8);
  t += 2 * al(nf2);
  t += 4 * al(2 * ndof * 8);
  t += al((size_t)adj_blocks * 2 * FR_MAX_MODES * 8);
  if (f->prm.vel.kind == FR_VEL_STREAM) {  // phase table and per-point velocity adjoint
    const size_t np = (size_t)f->E * (f->nu + f->nf);
    t += al(np * (size_t)f->prm.vel.n_modes * 2 * 8);
    t += al(np * 2 * 8);
  }
  z.total = t;
  return z;
}

}  // namespace

extern "C" int fr_adjoint_workspace_bytes(fr_field* f, int n_steps, int ckpt_every, size_t* bytes) {
  if (!f || !bytes || n_steps < 1 || ckpt_every < 1) return FR_EINVAL;
  AdjSet as;
  if (!adj_kernels(f, &as)) return FR_EUNSUPPORTED;
  const int nb = (int)((f->E + as.et - 1) / as.et);
  *bytes = sizes(f, n_steps, ckpt_every, nb).total;
  return FR_OK;
}

extern "C" int fr_adjoint_record(fr_field* f, int n_steps, int ckpt_every, void* ws, size_t ws_bytes,
                                 void* stream) {
  if (!f || !ws || n_steps < 1 || ckpt_every < 1) return FR_EINVAL;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return FR_EINVAL;
  if (f->prm.normal != FR_NORMAL_PSI) return FR_EUNSUPPORTED;  // adjoint of the preconditioned method only
  if (f->prm.wall != FR_WALL_COPY) return FR_EUNSUPPORTED;     // and of the paper's copy-ghost walls
  AdjSet as;
  if (!adj_kernels(f, &as)) return FR_EUNSUPPORTED;
  const int nb = (int)((f->E + as.et - 1) / as.et);
  const Sizes z = sizes(f, n_steps, ckpt_every, nb);
  if (ws_bytes < z.total) return FR_ENOMEM;
  // the recorded window must not contain a preconditioning step
  for (int64_t n = f->nstep; n < f->nstep + n_steps; ++n)
    if (n > 0 && n % f->prm.n_precond == 0) return FR_EUNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  AdjRecord& R = f->rec;
  R = AdjRecord();
  R.n_steps = n_steps;
  R.ckpt_every = ckpt_every;
  R.n_ckpt = z.n_ckpt;
  R.step0 = f->nstep;
  R.ws = reinterpret_cast<char*>(ws);
  R.bytes = ws_bytes;
  R.adj_blocks = nb;
  size_t off = 0;
  R.off_ckpt = off;
  off += (z.n_ckpt + 1) * z.ckpt_slot;
  R.off_stage = off;
  off += (size_t)ckpt_every * 4 * z.stage_slot;
  R.off_times = off;
  off += al((size_t)ckpt_every * 8);
  const size_t nf2 = al((size_t)f->E * 2 * f->nf * 8), nd2 = al(2 * (size_t)f->E * f->nu * 8);
  R.off_Y = off;
  off += nf2;
  R.off_lamuo = off;
  off += nf2;
  R.off_lamU = off;
  off += nd2;
  R.off_Lp = off;
  off += nd2;
  R.off_Lu = off;
  off += nd2;
  R.off_Lk = off;
  off += nd2;
  R.off_coefp = off;
  off += al((size_t)nb * 2 * FR_MAX_MODES * 8);
  if (f->prm.vel.kind == FR_VEL_STREAM) {
    const size_t np = (size_t)f->E * (f->nu + f->nf);
    R.off_cs = off;
    off += al(np * (size_t)f->prm.vel.n_modes * 2 * 8);
    R.off_lv = off;
  }
  const size_t ubytes = 2 * (size_t)f->E * f->nu * 8;
  for (int n = 0; n < n_steps; ++n) {
    if (n % ckpt_every == 0) {
      char* slot = R.ws + R.off_ckpt + (size_t)(n / ckpt_every) * z.ckpt_slot;
      CK(cudaMemcpyAsync(slot, f->args.u, ubytes, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(slot + ubytes, f->args.dstate + DS_TIME, 8, cudaMemcpyDeviceToDevice, s));
    }
    const int rc = field_run_step(f, s, false);
    if (rc) return rc;
  }
  char* last = R.ws + R.off_ckpt + (size_t)z.n_ckpt * z.ckpt_slot;
  CK(cudaMemcpyAsync(last, f->args.u, ubytes, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(last + ubytes, f->args.dstate + DS_TIME, 8, cudaMemcpyDeviceToDevice, s));
  R.active = 1;
  return FR_OK;
}

extern "C" int fr_adjoint_step(fr_field* f, const double* dJ_dphiT, const double* dJ_dpsiT, double* dJ_du0,
                               double* dJ_dcoef, void* stream) {
  if (!f || !dJ_dphiT || !dJ_du0) return FR_EINVAL;
  AdjRecord& R = f->rec;
  if (!R.active) return FR_EINVAL;
  AdjSet as;
  if (!adj_kernels(f, &as)) return FR_EUNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const Sizes z = sizes(f, R.n_steps, R.ckpt_every, R.adj_blocks);
  const int64_t E = f->E;
  const int NU = f->nu;
  const size_t ubytes = 2 * (size_t)E * NU * 8;
  double* Y = reinterpret_cast<double*>(R.ws + R.off_Y);
  double* lamuo = reinterpret_cast<double*>(R.ws + R.off_lamuo);
  double* lamU = reinterpret_cast<double*>(R.ws + R.off_lamU);
  double* Lp = reinterpret_cast<double*>(R.ws + R.off_Lp);
  double* Lu = reinterpret_cast<double*>(R.ws + R.off_Lu);
  double* Lk = reinterpret_cast<double*>(R.ws + R.off_Lk);
  double* coefp = reinterpret_cast<double*>(R.ws + R.off_coefp);
  double* times = reinterpret_cast<double*>(R.ws + R.off_times);
  const int M2 = f->prm.vel.kind == FR_VEL_STREAM ? 2 * f->args.cd.vel.n_modes : 0;
  const double dt = f->prm.dt;
  int grid = (int)((E * NU + 255) / 256);
  if (grid > 152 * 16) grid = 152 * 16;
  k_pack_lam<<<grid, 256, 0, s>>>(Lp, dJ_dphiT, dJ_dpsiT, E, NU);
  if (M2) CK(cudaMemsetAsync(coefp, 0, (size_t)R.adj_blocks * M2 * 8, s));
  double* cs = M2 ? reinterpret_cast<double*>(R.ws + R.off_cs) : nullptr;
  double* lv = M2 ? reinterpret_cast<double*>(R.ws + R.off_lv) : nullptr;
  if (M2) as.tab(f->args, cs, s);
  const int64_t npts = E * (f->nu + f->nf);
  const int64_t nstep_save = f->nstep;
  std::vector<double> th(R.ckpt_every);
  for (int seg = R.n_ckpt - 1; seg >= 0; --seg) {
    const int s0 = seg * R.ckpt_every;
    const int s1 = s0 + R.ckpt_every < R.n_steps ? s0 + R.ckpt_every : R.n_steps;
    // restore the checkpoint and recompute the segment, keeping the stage inputs
    char* slot = R.ws + R.off_ckpt + (size_t)seg * z.ckpt_slot;
    CK(cudaMemcpyAsync(f->args.u, slot, ubytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(f->args.dstate + DS_TIME, slot + ubytes, 8, cudaMemcpyDeviceToDevice, s));
    int rc = field_stage_and_traces(f, s);
    if (rc) return rc;
    f->nstep = R.step0 + s0;
    for (int n = s0; n < s1; ++n) {
      CK(cudaMemcpyAsync(times + (n - s0), f->args.dstate + DS_TIME, 8, cudaMemcpyDeviceToDevice, s));
      KArgs a = f->args;
      a.use_dev_time = 1;
      a.dt = dt;
      a.rk = rk_const(dt);
      for (int st = 1; st <= 4; ++st) {
        char* U = R.ws + R.off_stage + ((size_t)(n - s0) * 4 + (st - 1)) * z.stage_slot;
        CK(cudaMemcpyAsync(U, f->args.ustg, ubytes, cudaMemcpyDeviceToDevice, s));
        a.stage = st;
        f->ks.kb[0](a, s);
        f->ks.ka[0](a, s);
      }
      f->nstep++;
    }
    CK(cudaMemcpyAsync(th.data(), times, (size_t)(s1 - s0) * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // reverse through the segment
    for (int n = s1 - 1; n >= s0; --n) {
      for (int st = 4; st >= 1; --st) {
        AdjArgs B;
        std::memset(&B, 0, sizeof(B));
        B.K = f->args;
        B.K.ustg = R.ws + R.off_stage + ((size_t)(n - s0) * 4 + (st - 1)) * z.stage_slot;
        B.K.use_dev_time = 0;
        B.K.t = th[n - s0] + (st == 1 ? 0.0 : (st == 4 ? dt : 0.5 * dt));
        B.K.stage = 0;
        f->ks.ka[0](B.K, s);  // traces of this stage input
        B.lamk = st == 4 ? Lp : Lk;
        B.lam_scale = st == 4 ? dt / 6.0 : 1.0;
        B.Y = Y;
        B.lamU = lamU;
        B.lamuo = lamuo;
        B.coefp = coefp;
        B.want_coef = M2 > 0;
        B.lv = lv;
        B.Lp = Lp;
        B.Lu = Lu;
        B.first = st == 4;
        switch (st) {
          case 4: B.Lk = Lk; B.c_lp = dt / 3.0; B.c_a = dt; break;
          case 3: B.Lk = Lk; B.c_lp = dt / 3.0; B.c_a = 0.5 * dt; break;
          case 2: B.Lk = Lk; B.c_lp = dt / 6.0; B.c_a = 0.5 * dt; break;
          default: B.Lk = nullptr; B.c_lp = 0.0; B.c_a = 0.0;
        }
        as.a(B, s);
        as.b(B, s);
        if (M2) {
          const double T = f->prm.vel.T;
          const double gt = T > 0.0 ? std::cos(M_PI * B.K.t / T) : 1.0;  // time factor of this stage
          k_coef_acc<<<R.adj_blocks, 256, 0, s>>>(lv, cs, npts, f->args.cd.vel, gt, coefp);
        }
        // adj_c reads Lk (through lamk of the next stage) only after this stage
        // is complete; writing Lk here is safe because stage st consumed it in adj_a/adj_b
        as.c(B, s);
      }
      std::swap(Lp, Lu);
    }
  }
  CK(cudaGetLastError());
  k_unpack_lam<<<grid, 256, 0, s>>>(Lp, dJ_du0, E, NU);
  if (M2 && dJ_dcoef) k_coef_reduce<<<1, 64, 0, s>>>(coefp, R.adj_blocks, M2, dJ_dcoef);
  // leave the field at the end of the recorded window
  char* last = R.ws + R.off_ckpt + (size_t)z.n_ckpt * z.ckpt_slot;
  CK(cudaMemcpyAsync(f->args.u, last, ubytes, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(f->args.dstate + DS_TIME, last + ubytes, 8, cudaMemcpyDeviceToDevice, s));
  const int rc = field_stage_and_traces(f, s);
  if (rc) return rc;
  f->nstep = nstep_save;
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  return FR_OK;
}
