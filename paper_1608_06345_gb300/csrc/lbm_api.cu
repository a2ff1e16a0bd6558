// C ABI of the library (include/lbm.h): instance lifetime, validation,
// device memory layout and the launch sequences of init / step / moments /
// conservation sums.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/lbm.h"
#include "runtime.h"

namespace lbm {

// Second pass of the conservation sums: one warp per value, lane-strided
// sums over the block partials, then a shuffle tree (fixed order).
__global__ void k_conserve_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  // one warp per value, fixed order: lane-strided sums, then a shuffle tree
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k >= kRedVals) return;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += partial[b * kRedVals + k];
  s = warp_sum(s);
  if (lane == 0) out[k] = s;
}

int resolve_reference(int prec, double rho0, double T0, double* rho0_out, double* T0_out) {
  const bool s16 = (prec == kF32S16F || prec == kF32S16BF);
  double r;
  if (rho0 > 0.0 && std::isfinite(rho0)) {
    r = rho0;
  } else if (rho0 < 0.0) {
    if (s16) return LBM_EINVAL;  // the 16-bit codec scales by the reference
    r = 0.0;
  } else {  // 0 or NaN: the precision's default
    r = (prec == kF64) ? 0.0 : 1.0;
  }
  *rho0_out = r;
  *T0_out = (T0 > 0.0 && std::isfinite(T0)) ? T0 : 1.0;
  return LBM_OK;
}

// Reference equilibrium of the instance per velocity group, Eq. (18) at
// (rho0, u = 0, T0): gref = w rho0 (1 + pref) with
// pref = t0 (x2 - D)/2 + t0^2 [x2^2 - 2 (D + 2) x2 + D (D + 2)] / 8, t0 = T0 - 1;
// the 16-bit h codec scales by href = (delta/2) T0 gref (by gref if delta = 0).
void reference_constants(const LatticeTable& t, double delta, double rho0, double T0, double* gref,
                         double* pref, double* hscale) {
  const double D = t.D, th = T0 - 1.0;
  for (int g = 0; g < 10; ++g) {
    if (g >= t.G) {
      gref[g] = hscale[g] = 1.0;
      pref[g] = 0.0;
      continue;
    }
    const double x2 = t.x2g[g];
    pref[g] = 0.5 * th * (x2 - D) + 0.125 * th * th * (x2 * x2 - 2.0 * (D + 2.0) * x2 + D * (D + 2.0));
    gref[g] = t.wg[g] * rho0 * (1.0 + pref[g]);
    hscale[g] = (delta > 0.0) ? 0.5 * delta * T0 * gref[g] : gref[g];
  }
}

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(LBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t word_of(int prec) {
  switch (prec) {
    case kF64: return 8;
    case kF32: return 4;
    case kF32S16F:
    case kF32S16BF: return 2;
  }
  return 0;
}

// Validates lattice/grid; fills D, Q and the derived sizes.  Returns "" if ok.
std::string check_grid(int lattice, const lbm_grid* g, int* D, int* Q) {
  if (lattice != LBM_D2Q37 && lattice != LBM_D3Q107) return "unknown lattice";
  if (!g) return "grid is NULL";
  *D = (lattice == LBM_D2Q37) ? 2 : 3;
  *Q = (lattice == LBM_D2Q37) ? 37 : 107;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1) return "grid dimensions must be >= 1";
  if (*D == 2 && g->nz != 1) return "D2Q37 needs nz == 1";
  for (int a = 0; a < 3; ++a)
    if (g->bc[a] != LBM_PERIODIC && g->bc[a] != LBM_ZERO_GRADIENT) return "unknown boundary kind";
  if (word_of(g->prec) == 0) return "unknown precision";
  const long long N = (long long)g->nx * g->ny * g->nz;
  if (N > 0x7fffffffLL) return "more than 2^31-1 cells";
  if (g->ny > 65535 || g->nz > 65535) return "ny and nz must be <= 65535";
  return "";
}

size_t buffer_bytes(int Q, long long N, int prec) {
  const size_t ps = round_up((size_t)N, 64);
  return round_up(2 * (size_t)Q * ps * word_of(prec), 256);
}

template <class C>
void fill_args(const Instance& I, Args<C>* a) {
  std::memset(a, 0, sizeof(*a));
  for (int k = 0; k < 3; ++k) {
    a->n[k] = I.n[k];
    a->bc[k] = I.bc[k];
  }
  a->ps = I.ps;
  const double r = I.table.r;
  a->r = (C)r;
  a->half_r2 = (C)(0.5 * r * r);
  a->Dd = (C)(I.D + I.delta);
  a->inv_Dd = (C)(1.0 / (I.D + I.delta));
  a->half_delta = (C)(0.5 * I.delta);
  a->omega_f = (C)(1.0 / I.tau_f);
  a->omega_g = (C)(1.0 / I.tau_g);
  a->rho0 = (C)I.rho0;
  a->T0 = (C)I.T0;
  a->t0 = (C)(I.T0 - 1.0);
  double gref[10], pref[10], hscale[10];
  reference_constants(I.table, I.delta, I.rho0, I.T0, gref, pref, hscale);
  for (int g = 0; g < 10; ++g) {
    a->wg[g] = (C)I.table.wg[g];
    a->x2g[g] = (C)I.table.x2g[g];
    a->gref[g] = (C)gref[g];
    a->pref[g] = (C)pref[g];
    a->inv_gref[g] = (C)(gref[g] != 0.0 ? 1.0 / gref[g] : 0.0);  // 0: whole storage (16-bit codec unused)
    a->hscale[g] = (C)hscale[g];
    a->inv_hscale[g] = (C)(hscale[g] != 0.0 ? 1.0 / hscale[g] : 0.0);
  }
  a->flag = I.flag;
}

const Launchers& launchers_of(const Instance* I) { return launchers_for(I->lattice, I->prec); }
cudaError_t launch_step(const Instance* I, const void* src, void* dst) { return launchers_of(I).step(I, src, dst); }
cudaError_t launch_init(const Instance* I, void* dst, const double* rho, const double* u, const double* T) {
  return launchers_of(I).init(I, dst, rho, u, T);
}
cudaError_t launch_moments(const Instance* I, const void* src, double* rho, double* u, double* T) {
  return launchers_of(I).moments(I, src, rho, u, T);
}
cudaError_t launch_conserve(const Instance* I, const void* src, double* partial, int nblocks) {
  return launchers_of(I).conserve(I, src, partial, nblocks);
}

int reduction_blocks(long long N) {
  long long b = (N + kRedThreads - 1) / kRedThreads;
  if (b > kRedMaxBlocks) b = kRedMaxBlocks;
  if (b < 1) b = 1;
  return (int)b;
}

// Reads the error word (synchronising the stream) and maps it to a status.
int check_status(Instance* I) {
  unsigned int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, I->flag, sizeof(flag), cudaMemcpyDeviceToHost, I->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(I->stream);
  if (e != cudaSuccess) return cuda_fail(e, "synchronising the instance stream");
  if (flag & 1u) return fail(LBM_ENONFINITE, "a step met a non-finite density or temperature");
  return LBM_OK;
}

}  // namespace

int set_error(int code, const std::string& msg) { return fail(code, msg); }

StepShape default_shape(int lattice, int prec) {
  (void)lattice;
  (void)prec;
  return StepShape{0};
}


int prepare_instance(Instance* I, int lattice, double gamma, double tau_f, double tau_g, const lbm_grid* grid) {
  int D, Q;
  std::string msg = check_grid(lattice, grid, &D, &Q);
  if (!msg.empty()) return fail(LBM_EINVAL, msg);
  if (!(gamma > 1.0) || !std::isfinite(gamma)) return fail(LBM_EINVAL, "gamma must be > 1");
  double delta = 2.0 / (gamma - 1.0) - D;
  if (delta < -1e-12) return fail(LBM_EINVAL, "gamma gives delta < 0 (gamma must be <= (D+2)/D)");
  if (delta < 0.0) delta = 0.0;
  if (!(tau_f > 0.5) || !(tau_g > 0.5) || !std::isfinite(tau_f) || !std::isfinite(tau_g))
    return fail(LBM_EINVAL, "tau_f and tau_g must be > 0.5");
  I->lattice = lattice;
  I->prec = grid->prec;
  I->D = D;
  I->Q = Q;
  I->n[0] = grid->nx;
  I->n[1] = grid->ny;
  I->n[2] = grid->nz;
  for (int a = 0; a < 3; ++a) I->bc[a] = grid->bc[a];
  I->N = (long long)grid->nx * grid->ny * grid->nz;
  I->ps = (long long)round_up((size_t)I->N, 64);
  I->word = word_of(grid->prec);
  I->buf_bytes = buffer_bytes(Q, I->N, grid->prec);
  I->stream = static_cast<cudaStream_t>(grid->stream);
  I->gamma = gamma;
  I->delta = delta;
  I->tau_f = tau_f;
  I->tau_g = tau_g;
  if (resolve_reference(grid->prec, grid->rho0, grid->T0, &I->rho0, &I->T0) != LBM_OK)
    return fail(LBM_EINVAL, "16-bit storage needs a positive reference density rho0 (rho0 < 0 asks for whole storage)");
  I->shape = default_shape(lattice, grid->prec);
  I->fd_kernel = LBM_FD_AUTO;
  I->graph_steps = 64;
  I->graph_shape = -1;
  I->graph_exec = nullptr;
  I->graph = nullptr;
  if (build_lattice_table(lattice, &I->table) != 0) return fail(LBM_EINVAL, "lattice table refinement failed");
  I->G = I->table.G;
  return LBM_OK;
}

void fill_instance_args(Instance* I) {
  fill_args(*I, &I->ad);
  fill_args(*I, &I->af);
}

size_t instance_buffer_bytes(int Q, long long N, int prec) { return buffer_bytes(Q, N, prec); }

const Launchers& launchers_for(int lattice, int prec) {
  static const Launchers* table[2][4] = {{&kLaunchers_0_0, &kLaunchers_0_1, &kLaunchers_0_2, &kLaunchers_0_3},
                                         {&kLaunchers_1_0, &kLaunchers_1_1, &kLaunchers_1_2, &kLaunchers_1_3}};
  return *table[lattice][prec];
}

void drop_graph(Instance* I) {
  if (I->graph_exec) cudaGraphExecDestroy(I->graph_exec);
  if (I->graph) cudaGraphDestroy(I->graph);
  I->graph_exec = nullptr;
  I->graph = nullptr;
  I->graph_shape = -1;
}

// Capture graph_steps steps starting from buffer cur (on a private stream:
// the legacy default stream cannot be captured); the instance's stream
// then replays it.
cudaError_t capture_graph(Instance* I) {
  drop_graph(I);
  cudaError_t e = launchers_of(I).configure(I);
  if (e != cudaSuccess) return e;
  cudaStream_t cs;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaStream_t keep = I->stream;
  I->stream = cs;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  cudaError_t le = cudaSuccess;
  if (e == cudaSuccess) {
    int c = I->cur;
    for (int k = 0; k < I->graph_steps && le == cudaSuccess; ++k) {
      le = launch_step(I, I->buf[c], I->buf[1 - c]);
      c ^= 1;
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess && le == cudaSuccess) {
      e = cudaGraphInstantiate(&I->graph_exec, g, 0);
      if (e == cudaSuccess) I->graph = g;
      else cudaGraphDestroy(g);
    } else if (g) {
      cudaGraphDestroy(g);
    }
  }
  I->stream = keep;
  cudaStreamDestroy(cs);
  if (le != cudaSuccess) return le;
  if (e == cudaSuccess) I->graph_shape = I->shape.index;
  return e;
}

}  // namespace lbm

// The opaque handle type of the C ABI is the runtime's instance record.
struct lbm_instance : public lbm::Instance {};

using namespace lbm;

extern "C" {

size_t lbm_state_bytes(int lattice, const lbm_grid* grid) {
  int D, Q;
  if (!check_grid(lattice, grid, &D, &Q).empty()) return 0;
  const long long N = (long long)grid->nx * grid->ny * grid->nz;
  return 2 * buffer_bytes(Q, N, grid->prec) + kTailBytes;
}

int lbm_create(lbm_handle* out, int lattice, double gamma, double tau_f, double tau_g, const lbm_grid* grid) {
  if (!out) return fail(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  lbm_instance* I = new (std::nothrow) lbm_instance();
  if (!I) return fail(LBM_ENOMEM, "host allocation failed");
  int rc = prepare_instance(I, lattice, gamma, tau_f, tau_g, grid);
  if (rc != LBM_OK) {
    delete I;
    return rc;
  }

  const size_t need = 2 * I->buf_bytes + kTailBytes;
  if (grid->device_mem) {
    if (grid->device_bytes < need) {
      delete I;
      return fail(LBM_ENOMEM, "device_mem is smaller than lbm_state_bytes()");
    }
    if (reinterpret_cast<uintptr_t>(grid->device_mem) % 256 != 0) {
      delete I;
      return fail(LBM_EINVAL, "device_mem must be 256-byte aligned");
    }
    I->mem = static_cast<unsigned char*>(grid->device_mem);
    I->own_mem = false;
  } else {
    cudaError_t e = cudaMalloc(&I->mem, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete I;
      return fail(LBM_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    I->own_mem = true;
  }
  I->buf[0] = I->mem;
  I->buf[1] = I->mem + I->buf_bytes;
  unsigned char* tail = I->mem + 2 * I->buf_bytes;
  I->flag = reinterpret_cast<unsigned int*>(tail);
  I->red_out = reinterpret_cast<double*>(tail + 256);
  I->red_partial = reinterpret_cast<double*>(tail + 512);
  I->cur = 0;
  fill_instance_args(I);
  cudaError_t e = cudaMemsetAsync(tail, 0, kTailBytes, I->stream);
  if (e != cudaSuccess) {
    if (I->own_mem) cudaFree(I->mem);
    delete I;
    return cuda_fail(e, "clearing the instance tail");
  }
  *out = I;
  return LBM_OK;
}

int lbm_destroy(lbm_handle h) {
  if (!h) return LBM_OK;
  lbm_instance* I = h;
  int rc = LBM_OK;
  if (I->graph_exec) {
    cudaStreamSynchronize(I->stream);
    drop_graph(I);
  }
  if (I->own_mem) {
    cudaError_t e = cudaStreamSynchronize(I->stream);
    if (e == cudaSuccess) e = cudaFree(I->mem);
    if (e != cudaSuccess) rc = cuda_fail(e, "freeing the instance");
  }
  delete I;
  return rc;
}

int lbm_init_device(lbm_handle h, const double* rho, const double* u, const double* T) {
  if (!h) return fail(LBM_EINVAL, "handle is NULL");
  if (h->N > 0 && (!rho || !u || !T)) return fail(LBM_EINVAL, "field pointer is NULL");
  cudaError_t e = launch_init(h, h->buf[h->cur], rho, u, T);
  if (e != cudaSuccess) return cuda_fail(e, "launching init");
  h->steps_done = 0;
  return LBM_OK;
}

int lbm_init(lbm_handle h, const double* rho, const double* u, const double* T) {
  if (!h) return fail(LBM_EINVAL, "handle is NULL");
  if (h->N > 0 && (!rho || !u || !T)) return fail(LBM_EINVAL, "field pointer is NULL");
  // stage the FP64 fields in the idle buffer (it always has room: 2Q words
  // per cell >= (D + 2) doubles per cell)
  double* st = static_cast<double*>(h->buf[1 - h->cur]);
  const size_t nb = sizeof(double) * (size_t)h->N;
  cudaError_t e = cudaMemcpyAsync(st, rho, nb, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(st + h->N, u, nb * h->D, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(st + (1 + h->D) * h->N, T, nb, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copying the initial fields");
  int rc = lbm_init_device(h, st, st + h->N, st + (1 + h->D) * h->N);
  if (rc != LBM_OK) return rc;
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "synchronising after init");
  return LBM_OK;
}

int lbm_step(lbm_handle h, long n) {
  if (!h) return fail(LBM_EINVAL, "handle is NULL");
  if (n < 0) return fail(LBM_EINVAL, "n must be >= 0");
  if (h->N == 0) return LBM_OK;
  // whole bundles as graph replays (the graph's even step count leaves cur
  // unchanged; it is captured from the current parity, so recapture if the
  // shape changed), the remainder as plain launches
  if (h->graph_steps > 0 && n >= 2L * h->graph_steps) {
    if (!h->graph_exec || h->graph_shape != h->shape.index || h->cur != 0) {
      // the graph is captured with buffer 0 current: step once if needed
      if (h->cur != 0) {
        cudaError_t e = launch_step(h, h->buf[h->cur], h->buf[1 - h->cur]);
        if (e != cudaSuccess) return cuda_fail(e, "launching the step kernel");
        h->cur ^= 1;
        ++h->steps_done;
        --n;
      }
      if (!h->graph_exec || h->graph_shape != h->shape.index) {
        cudaError_t e = capture_graph(h);
        if (e != cudaSuccess) return cuda_fail(e, "capturing the step graph");
      }
    }
    while (n >= h->graph_steps) {
      cudaError_t e = cudaGraphLaunch(h->graph_exec, h->stream);
      if (e != cudaSuccess) return cuda_fail(e, "launching the step graph");
      n -= h->graph_steps;
      h->steps_done += h->graph_steps;
    }
  }
  for (long k = 0; k < n; ++k) {
    cudaError_t e = launch_step(h, h->buf[h->cur], h->buf[1 - h->cur]);
    if (e != cudaSuccess) return cuda_fail(e, "launching the step kernel");
    h->cur ^= 1;
    ++h->steps_done;
  }
  return LBM_OK;
}

int lbm_set_fd_kernel(lbm_handle h, int kernel) {
  if (!h) return fail(LBM_EINVAL, "handle is NULL");
  if (kernel != LBM_FD_AUTO && kernel != LBM_FD_CELL && kernel != LBM_FD_MARCH)
    return fail(LBM_EINVAL, "kernel must be LBM_FD_AUTO, LBM_FD_CELL or LBM_FD_MARCH");
  if (kernel == LBM_FD_MARCH && h->D != 2) return fail(LBM_EINVAL, "the marched finite-difference step is 2D only");
  h->fd_kernel = kernel;
  return LBM_OK;
}

int lbm_step_fd(lbm_handle h, long n, double lambda) {
  if (!h) return fail(LBM_EINVAL, "handle is NULL");
  if (n < 0) return fail(LBM_EINVAL, "n must be >= 0");
  if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail(LBM_EINVAL, "lambda = dt/dx must be > 0");
  if (h->N == 0) return LBM_OK;
  for (long k = 0; k < n; ++k) {
    cudaError_t e = launchers_of(h).step_fd(h, h->buf[h->cur], h->buf[1 - h->cur], lambda);
    if (e != cudaSuccess) return cuda_fail(e, "launching the finite-difference step");
    h->cur ^= 1;
    ++h->steps_done;
  }
  return LBM_OK;
}

int lbm_moments_device(lbm_handle h, double* rho, double* u, double* T) {
  if (!h) return fail(LBM_EINVAL, "handle is NULL");
  if (h->N > 0 && (!rho || !u || !T)) return fail(LBM_EINVAL, "field pointer is NULL");
  cudaError_t e = launch_moments(h, h->buf[h->cur], rho, u, T);
  if (e != cudaSuccess) return cuda_fail(e, "launching moments");
  return LBM_OK;
}

int lbm_moments(lbm_handle h, double* rho, double* u, double* T) {
  if (!h) return fail(LBM_EINVAL, "handle is NULL");
  if (h->N > 0 && (!rho || !u || !T)) return fail(LBM_EINVAL, "field pointer is NULL");
  double* st = static_cast<double*>(h->buf[1 - h->cur]);
  int rc = lbm_moments_device(h, st, st + h->N, st + (1 + h->D) * h->N);
  if (rc != LBM_OK) return rc;
  const size_t nb = sizeof(double) * (size_t)h->N;
  cudaError_t e = cudaMemcpyAsync(rho, st, nb, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(u, st + h->N, nb * h->D, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(T, st + (1 + h->D) * h->N, nb, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copying moments to the host");
  return check_status(h);
}

int lbm_conserved(lbm_handle h, double* out) {
  if (!h) return fail(LBM_EINVAL, "handle is NULL");
  if (!out) return fail(LBM_EINVAL, "out is NULL");
  const int nb = reduction_blocks(h->N);
  cudaError_t e = cudaSuccess;
  if (h->N > 0) {
    e = launch_conserve(h, h->buf[h->cur], h->red_partial, nb);
    if (e == cudaSuccess) {
      k_conserve_final<<<1, 32 * kRedVals, 0, h->stream>>>(h->red_partial, nb, h->red_out);
      e = cudaGetLastError();
    }
  } else {
    e = cudaMemsetAsync(h->red_out, 0, sizeof(double) * kRedVals, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "launching the conservation sums");
  double tmp[kRedVals];
  e = cudaMemcpyAsync(tmp, h->red_out, sizeof(tmp), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copying conservation sums");
  int rc = check_status(h);
  // the kernels sum deviations; add the reference totals
  const double Nd = (double)h->N;
  out[0] = Nd * h->rho0 + tmp[0];
  for (int a = 0; a < h->D; ++a) out[1 + a] = tmp[1 + a];
  out[1 + h->D] = Nd * h->rho0 * 0.5 * (h->D + h->delta) * h->T0 + tmp[4];
  return rc;
}

int lbm_sync(lbm_handle h) {
  if (!h) return fail(LBM_EINVAL, "handle is NULL");
  return check_status(h);
}

long lbm_steps_done(lbm_handle h) { return h ? h->steps_done : -1; }

size_t lbm_raw_state_bytes(lbm_handle h) {
  if (!h) return 0;
  return 2 * (size_t)h->Q * (size_t)h->N * h->word;
}

int lbm_get_state(lbm_handle h, void* host, size_t bytes) {
  if (!h || !host) return fail(LBM_EINVAL, "NULL argument");
  if (bytes < lbm_raw_state_bytes(h)) return fail(LBM_EINVAL, "host buffer too small");
  // 16-bit storage keeps (g_i, h_i) as one 4-byte pair: Q planes of pairs
  const bool paired = (h->prec == kF32S16F || h->prec == kF32S16BF);
  const size_t elem = paired ? 2 * h->word : h->word;
  const int planes = paired ? h->Q : 2 * h->Q;
  const size_t plane = (size_t)h->N * elem;
  unsigned char* dst = static_cast<unsigned char*>(host);
  const unsigned char* src = static_cast<const unsigned char*>(h->buf[h->cur]);
  cudaError_t e = cudaMemcpy2DAsync(dst, plane, src, (size_t)h->ps * elem, plane, planes, cudaMemcpyDeviceToHost,
                                    h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copying the state to the host");
  return LBM_OK;
}

int lbm_set_state(lbm_handle h, const void* host, size_t bytes) {
  if (!h || !host) return fail(LBM_EINVAL, "NULL argument");
  if (bytes < lbm_raw_state_bytes(h)) return fail(LBM_EINVAL, "host buffer too small");
  const bool paired = (h->prec == kF32S16F || h->prec == kF32S16BF);
  const size_t elem = paired ? 2 * h->word : h->word;
  const int planes = paired ? h->Q : 2 * h->Q;
  const size_t plane = (size_t)h->N * elem;
  unsigned char* dst = static_cast<unsigned char*>(h->buf[h->cur]);
  cudaError_t e = cudaMemcpy2DAsync(dst, (size_t)h->ps * elem, host, plane, plane, planes, cudaMemcpyHostToDevice,
                                    h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copying the state to the device");
  return LBM_OK;
}

int lbm_lattice_table(int lattice, int* q, int* c, double* w, double* r) {
  LatticeTable t;
  if (build_lattice_table(lattice, &t) != 0) return fail(LBM_EINVAL, "unknown lattice");
  const LatticeDef& L = (lattice == LBM_D2Q37) ? kD2Q37 : kD3Q107;
  if (q) *q = L.Q;
  for (int i = 0; i < L.Q; ++i) {
    if (c)
      for (int a = 0; a < L.D; ++a) c[i * L.D + a] = L.c[i][a];
    if (w) w[i] = t.wg[L.grp[i]];
  }
  if (r) *r = t.r;
  return LBM_OK;
}

int lbm_shape_info(int lattice, int prec, int index, int* stage, int* block) {
  if (lattice != LBM_D2Q37 && lattice != LBM_D3Q107) return fail(LBM_EINVAL, "unknown lattice");
  if (prec < kF64 || prec > kF32S16BF) return fail(LBM_EINVAL, "unknown precision");
  const Launchers& L = launchers_for(lattice, prec);
  if (index < 0 || index >= L.shape_count()) return fail(LBM_EINVAL, "shape index out of range");
  int st = 0, bx = 0;
  L.shape_get(index, &st, &bx);
  if (stage) *stage = st;
  if (block) *block = bx;
  return LBM_OK;
}

int lbm_set_shape(lbm_handle h, int index) {
  if (!h) return fail(LBM_EINVAL, "handle is NULL");
  if (index < 0 || index >= launchers_of(h).shape_count()) return fail(LBM_EINVAL, "shape index out of range");
  h->shape.index = index;
  return LBM_OK;
}

int lbm_get_shape(lbm_handle h) { return h ? h->shape.index : -1; }

int lbm_set_graph_steps(lbm_handle h, int steps) {
  if (!h) return fail(LBM_EINVAL, "handle is NULL");
  if (steps < 0 || steps % 2 != 0 || steps > 4096) return fail(LBM_EINVAL, "graph steps must be even, 0..4096");
  if (steps != h->graph_steps) {
    cudaStreamSynchronize(h->stream);
    drop_graph(h);
    h->graph_steps = steps;
  }
  return LBM_OK;
}

int lbm_autotune(lbm_handle h, int reps, int* best_index, double* best_us) {
  if (!h) return fail(LBM_EINVAL, "handle is NULL");
  if (reps < 1) return fail(LBM_EINVAL, "reps must be >= 1");
  if (h->N == 0) {
    if (best_index) *best_index = h->shape.index;
    if (best_us) *best_us = 0.0;
    return LBM_OK;
  }
  // every trial reads the current buffer and writes the idle one without
  // swapping them, so the state is not changed
  const int n = launchers_of(h).shape_count();
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(e, "creating tuning events");
  const int keep = h->shape.index;
  int best = keep;
  float best_ms = 0.f;
  for (int k = 0; k < n && e == cudaSuccess; ++k) {
    h->shape.index = k;
    for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = launch_step(h, h->buf[h->cur], h->buf[1 - h->cur]);
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_step(h, h->buf[h->cur], h->buf[1 - h->cur]);
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (k == 0 || ms < best_ms)) {
      best_ms = ms;
      best = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    h->shape.index = keep;
    return cuda_fail(e, "autotuning the step");
  }
  h->shape.index = best;
  if (best_index) *best_index = best;
  if (best_us) *best_us = 1e3 * best_ms / reps;
  return LBM_OK;
}

int lbm_quadrature(int D, int ngroups, const int* reps, int nconds, const int* exps, double r_in, int* q,
                   double* w_group, double* r, double* max_residual) {
  const int rc = hermite_quadrature(D, ngroups, reps, nconds, exps, r_in, q, w_group, r, max_residual);
  switch (rc) {
    case 0: return LBM_OK;
    case -1: return fail(LBM_EINVAL, "invalid arguments (D in 1..3, even exponents, r_in > 0, non-NULL arrays)");
    case -2: return fail(LBM_EINVAL, "a group representative generates no velocity");
    case -3: return fail(LBM_EINVAL, "the moment conditions are singular for these groups at r_in");
    case -4: return fail(LBM_EINVAL, "no scale r satisfies the conditions near r_in");
    default: return fail(LBM_EINVAL, "need ngroups (r fixed) or ngroups + 1 (r solved) conditions");
  }
}

const char* lbm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
