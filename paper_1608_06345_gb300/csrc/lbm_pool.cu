// Continuous-batching pool (lbm_pool_* in include/lbm.h): many independent
// instances of one lattice and precision resident in one device arena and
// advanced together, one batched launch per time step.
//
// Device memory of a pool, in one allocation (or the caller's device_mem):
//   [arena: budget_bytes, instance states carved out first-fit]
//   [slot descriptors: max_instances x PoolSlot<C>]
//   [tile list: max_tiles x int4 (slot, x0, y, z)] [tile count] [error words]
// A step bundle (bundle_steps x {batched step, advance}) is captured once as a
// CUDA graph; between bundles the host admits and retires instances by
// editing the slot table and the tile list, which the graph reads from
// device memory.
//
// Admissions may overlap a running bundle: the fields are copied and the
// instance initialised on a second (io) stream, in arena memory and a slot
// that no resident instance uses, and its error word is cleared there (only
// kernels of instances with steps left write error words).  The slot
// descriptor is written on the pool stream at the next lbm_pool_run, because
// the bundle's advance kernel walks every slot descriptor.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/lbm.h"
#include "runtime.h"

namespace lbm {
namespace {

struct Slot {
  bool used = false;
  bool desc_pending = false;  // descriptor not yet in device memory (written by the next run)
  alignas(16) unsigned char desc[sizeof(PoolSlot<double>)];
  long long ticket = -1;
  size_t off = 0, bytes = 0;  // arena range
  Instance inst;              // geometry, constants, buffers
  long steps_total = 0;
  long steps_done = 0;        // host mirror: steps enqueued so far
  bool nonfinite = false;     // error word seen at a sync point
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Stride of the slot table: exactly the struct size, because the kernels
// index it as an array of PoolSlot<C>.
size_t slot_bytes_of(int prec) { return prec == kF64 ? sizeof(PoolSlot<double>) : sizeof(PoolSlot<float>); }
static_assert(sizeof(PoolSlot<float>) % alignof(PoolSlot<float>) == 0, "slot stride");
static_assert(sizeof(PoolSlot<double>) % alignof(PoolSlot<double>) == 0, "slot stride");

}  // namespace
}  // namespace lbm

using namespace lbm;

struct lbm_pool {
  int lattice = 0, prec = 0, D = 2, Q = 37;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t io = nullptr;      // admissions (may overlap a running bundle)
  cudaEvent_t io_done = nullptr;  // recorded after the admissions' work
  unsigned char* mem = nullptr;
  bool own_mem = false;
  unsigned char* arena = nullptr;
  size_t arena_bytes = 0;
  unsigned char* d_slots = nullptr;
  size_t slot_size = 0;
  int max_slots = 0;
  int4* d_tiles = nullptr;
  int* d_ntiles = nullptr;
  int max_tiles = 0;
  unsigned int* d_flags = nullptr;
  const Launchers* L = nullptr;
  int grid = 0, tile_cells = 0, bundle_steps = 0;
  std::vector<Slot> slots;
  std::map<size_t, size_t> free_blocks;  // offset -> size
  std::unordered_map<long long, int> ticket_slot;
  long long next_ticket = 1;
  bool tiles_dirty = true;
  int ntiles_host = 0;
  size_t used_bytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<unsigned int> h_flags;
};

namespace {

struct PoolLayout {
  size_t arena, slots, tiles, ntiles, flags, total;
};

PoolLayout layout_of(int prec, size_t budget, int max_slots, int max_tiles) {
  PoolLayout l{};
  l.arena = 0;
  l.slots = align256(budget);
  l.tiles = l.slots + align256(slot_bytes_of(prec) * (size_t)max_slots);
  l.ntiles = l.tiles + align256(sizeof(int4) * (size_t)max_tiles);
  l.flags = l.ntiles + 256;
  l.total = l.flags + align256(sizeof(unsigned int) * (size_t)max_slots);
  return l;
}

int default_max_tiles(int lattice, int prec, size_t budget, int max_slots) {
  // a tile holds up to tile_cells cells; rows shorter than a tile still take
  // one: budget / (bytes per cell * 32) + 64 rows per instance covers both
  const size_t word = (prec == kF64) ? 8 : (prec == kF32 ? 4 : 2);
  const size_t Q = (lattice == LBM_D2Q37) ? 37 : 107;
  const size_t cell = 2 * 2 * Q * word;
  size_t t = budget / (cell * 32) + 64 * (size_t)max_slots;
  if (t > (size_t)1 << 26) t = (size_t)1 << 26;
  return (int)t;
}

bool arena_alloc(lbm_pool* p, size_t bytes, size_t* off) {
  for (auto it = p->free_blocks.begin(); it != p->free_blocks.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t roff = it->first + bytes;
      p->free_blocks.erase(it);
      if (rest) p->free_blocks[roff] = rest;
      return true;
    }
  }
  return false;
}

void arena_free(lbm_pool* p, size_t off, size_t bytes) {
  auto it = p->free_blocks.emplace(off, bytes).first;
  auto next = std::next(it);
  if (next != p->free_blocks.end() && it->first + it->second == next->first) {
    it->second += next->second;
    p->free_blocks.erase(next);
  }
  if (it != p->free_blocks.begin()) {
    auto prev = std::prev(it);
    if (prev->first + prev->second == it->first) {
      prev->second += it->second;
      p->free_blocks.erase(it);
    }
  }
}

int tiles_of(const lbm_pool* p, const Instance& I) {
  const long long per_row = (I.n[0] + p->tile_cells - 1) / p->tile_cells;
  return (int)(per_row * I.n[1] * I.n[2]);
}

int upload_tiles(lbm_pool* p) {
  std::vector<int4> h;
  h.reserve(p->ntiles_host);
  for (int s = 0; s < (int)p->slots.size(); ++s) {
    const Slot& sl = p->slots[s];
    if (!sl.used) continue;
    const Instance& I = sl.inst;
    for (int z = 0; z < I.n[2]; ++z)
      for (int y = 0; y < I.n[1]; ++y)
        for (int x0 = 0; x0 < I.n[0]; x0 += p->tile_cells) h.push_back(make_int4(s, x0, y, z));
  }
  const int n = (int)h.size();
  cudaError_t e = cudaSuccess;
  if (n) e = cudaMemcpyAsync(p->d_tiles, h.data(), sizeof(int4) * n, cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_ntiles, &n, sizeof(int), cudaMemcpyHostToDevice, p->stream);
  // the sources are host stack/heap memory: wait for the copies before they go away
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return set_error(LBM_ECUDA, std::string("uploading the tile list: ") + cudaGetErrorString(e));
  p->ntiles_host = n;
  p->tiles_dirty = false;
  return LBM_OK;
}

template <class C>
void make_slot_desc(const Instance& I, long steps, PoolSlot<C>* d) {
  std::memset(d, 0, sizeof(*d));
  if constexpr (std::is_same<C, double>::value) d->a = I.ad;
  else d->a = I.af;
  d->buf[0] = I.buf[0];
  d->buf[1] = I.buf[1];
  d->cur = 0;
  d->steps_left = (int)steps;
}

int build_graph(lbm_pool* p) {
  PoolLaunch pl{p->d_slots, p->d_tiles, p->d_ntiles, p->max_slots, p->grid, p->stream};
  cudaError_t e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return set_error(LBM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  cudaError_t le = cudaSuccess;
  for (int k = 0; k < p->bundle_steps && le == cudaSuccess; ++k) {
    le = p->L->pool_step(pl);
    if (le == cudaSuccess) le = p->L->pool_advance(pl);
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(p->stream, &g);
  if (le != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return set_error(LBM_ECUDA, std::string("capturing the step bundle: ") +
                                    cudaGetErrorString(le != cudaSuccess ? le : e));
  }
  e = cudaGraphInstantiate(&p->exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return set_error(LBM_ECUDA, std::string("instantiating the step bundle: ") + cudaGetErrorString(e));
  }
  p->graph = g;
  return LBM_OK;
}

void release(lbm_pool* p) {
  if (p->io) cudaStreamSynchronize(p->io);
  if (p->stream) cudaStreamSynchronize(p->stream);
  if (p->io_done) cudaEventDestroy(p->io_done);
  if (p->io) cudaStreamDestroy(p->io);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->own_mem && p->mem) cudaFree(p->mem);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

}  // namespace

extern "C" {

size_t lbm_pool_bytes(const lbm_pool_config* cfg) {
  if (!cfg || (cfg->lattice != LBM_D2Q37 && cfg->lattice != LBM_D3Q107) || cfg->prec < 0 || cfg->prec > 3 ||
      cfg->max_instances < 1)
    return 0;
  const int mt = cfg->max_tiles > 0 ? cfg->max_tiles
                                    : default_max_tiles(cfg->lattice, cfg->prec, cfg->budget_bytes, cfg->max_instances);
  return layout_of(cfg->prec, cfg->budget_bytes, cfg->max_instances, mt).total;
}

int lbm_pool_create(lbm_pool_handle* out, const lbm_pool_config* cfg) {
  if (!out || !cfg) return set_error(LBM_EINVAL, "NULL argument");
  *out = nullptr;
  if (cfg->lattice != LBM_D2Q37 && cfg->lattice != LBM_D3Q107) return set_error(LBM_EINVAL, "unknown lattice");
  if (cfg->prec < 0 || cfg->prec > 3) return set_error(LBM_EINVAL, "unknown precision");
  if (cfg->max_instances < 1 || cfg->max_instances > (1 << 20)) return set_error(LBM_EINVAL, "max_instances out of range");
  if (cfg->bundle_steps < 1 || cfg->bundle_steps > 4096) return set_error(LBM_EINVAL, "bundle_steps must be in [1, 4096]");
  if (cfg->budget_bytes < 256) return set_error(LBM_EINVAL, "budget_bytes too small");
  lbm_pool* p = new (std::nothrow) lbm_pool();
  if (!p) return set_error(LBM_ENOMEM, "host allocation failed");
  p->lattice = cfg->lattice;
  p->prec = cfg->prec;
  p->D = (cfg->lattice == LBM_D2Q37) ? 2 : 3;
  p->Q = (cfg->lattice == LBM_D2Q37) ? 37 : 107;
  p->L = &launchers_for(cfg->lattice, cfg->prec);
  p->tile_cells = p->L->pool_tile_cells;
  p->bundle_steps = cfg->bundle_steps;
  p->max_slots = cfg->max_instances;
  p->max_tiles = cfg->max_tiles > 0 ? cfg->max_tiles
                                    : default_max_tiles(cfg->lattice, cfg->prec, cfg->budget_bytes, cfg->max_instances);
  p->slot_size = slot_bytes_of(cfg->prec);
  const PoolLayout l = layout_of(cfg->prec, cfg->budget_bytes, p->max_slots, p->max_tiles);
  if (cfg->stream) {
    p->stream = static_cast<cudaStream_t>(cfg->stream);
  } else {
    // graphs cannot be captured on the legacy default stream
    cudaError_t e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete p;
      return set_error(LBM_ECUDA, std::string("creating the pool stream: ") + cudaGetErrorString(e));
    }
    p->own_stream = true;
  }
  {
    cudaError_t e = cudaStreamCreateWithFlags(&p->io, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->io_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      release(p);
      return set_error(LBM_ECUDA, std::string("creating the admission stream: ") + cudaGetErrorString(e));
    }
  }
  if (cfg->device_mem) {
    if (cfg->device_bytes < l.total) {
      release(p);
      return set_error(LBM_ENOMEM, "device_mem is smaller than lbm_pool_bytes()");
    }
    if (reinterpret_cast<uintptr_t>(cfg->device_mem) % 256 != 0) {
      release(p);
      return set_error(LBM_EINVAL, "device_mem must be 256-byte aligned");
    }
    p->mem = static_cast<unsigned char*>(cfg->device_mem);
  } else {
    cudaError_t e = cudaMalloc(&p->mem, l.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      release(p);
      return set_error(LBM_ENOMEM, std::string("cudaMalloc of the pool failed: ") + cudaGetErrorString(e));
    }
    p->own_mem = true;
  }
  p->arena = p->mem + l.arena;
  p->arena_bytes = cfg->budget_bytes / 256 * 256;
  p->d_slots = p->mem + l.slots;
  p->d_tiles = reinterpret_cast<int4*>(p->mem + l.tiles);
  p->d_ntiles = reinterpret_cast<int*>(p->mem + l.ntiles);
  p->d_flags = reinterpret_cast<unsigned int*>(p->mem + l.flags);
  p->slots.resize(p->max_slots);
  p->free_blocks[0] = p->arena_bytes;
  cudaError_t e = cudaMemsetAsync(p->mem + l.slots, 0, l.total - l.slots, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) {
    release(p);
    return set_error(LBM_ECUDA, std::string("clearing the pool tables: ") + cudaGetErrorString(e));
  }
  p->grid = p->L->pool_grid();
  if (p->grid <= 0) {
    release(p);
    return set_error(LBM_ECUDA, "could not size the persistent grid");
  }
  int rc = build_graph(p);
  if (rc != LBM_OK) {
    release(p);
    return rc;
  }
  p->tiles_dirty = true;
  *out = p;
  return LBM_OK;
}

int lbm_pool_destroy(lbm_pool_handle p) {
  if (!p) return LBM_OK;
  release(p);
  return LBM_OK;
}

size_t lbm_pool_instance_bytes(lbm_pool_handle p, const lbm_grid* grid) {
  if (!p || !grid) return 0;
  const long long N = (long long)grid->nx * grid->ny * grid->nz;
  if (N <= 0) return 0;
  return 2 * instance_buffer_bytes(p->Q, N, p->prec);
}

int lbm_pool_submit(lbm_pool_handle p, double gamma, double tau_f, double tau_g, const lbm_grid* grid,
                    const double* rho, const double* u, const double* T, long steps, long long* ticket) {
  if (!p || !grid || !ticket) return set_error(LBM_EINVAL, "NULL argument");
  if (steps < 0 || steps > 0x7fffffffL) return set_error(LBM_EINVAL, "steps out of range");
  if (grid->prec != p->prec) return set_error(LBM_EINVAL, "grid precision differs from the pool's");
  lbm_grid g = *grid;
  g.stream = p->stream;
  Instance I;
  int rc = prepare_instance(&I, p->lattice, gamma, tau_f, tau_g, &g);
  if (rc != LBM_OK) return rc;
  if (I.N > 0 && (!rho || !u || !T)) return set_error(LBM_EINVAL, "field pointer is NULL");
  int s = -1;
  for (int k = 0; k < p->max_slots; ++k)
    if (!p->slots[k].used) {
      s = k;
      break;
    }
  if (s < 0) return set_error(LBM_EBUSY, "all instance slots are in use");
  const size_t bytes = 2 * I.buf_bytes;
  const int nt = tiles_of(p, I);
  if (p->ntiles_host + nt > p->max_tiles) return set_error(LBM_EBUSY, "the tile list is full");
  size_t off = 0;
  if (!arena_alloc(p, bytes, &off)) return set_error(LBM_EBUSY, "the memory budget is full");
  I.mem = p->arena + off;
  I.own_mem = false;
  I.buf[0] = I.mem;
  I.buf[1] = I.mem + I.buf_bytes;
  I.cur = 0;
  I.flag = p->d_flags + s;
  I.red_out = nullptr;
  I.red_partial = nullptr;
  fill_instance_args(&I);

  // fields -> the idle buffer -> equilibrium in buffer 0, on the io stream
  // (this memory and this slot are not touched by a bundle in flight)
  I.stream = p->io;
  cudaError_t e = cudaSuccess;
  if (I.N > 0) {
    double* st = static_cast<double*>(I.buf[1]);
    const size_t nb = sizeof(double) * (size_t)I.N;
    e = cudaMemcpyAsync(st, rho, nb, cudaMemcpyHostToDevice, p->io);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st + I.N, u, nb * I.D, cudaMemcpyHostToDevice, p->io);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st + (1 + I.D) * I.N, T, nb, cudaMemcpyHostToDevice, p->io);
    if (e == cudaSuccess) e = p->L->init(&I, I.buf[0], st, st + I.N, st + (1 + I.D) * I.N);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(p->d_flags + s, 0, sizeof(unsigned int), p->io);
  if (e == cudaSuccess) e = cudaEventRecord(p->io_done, p->io);
  // the host fields must outlive the copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->io);
  I.stream = p->stream;
  if (e != cudaSuccess) {
    arena_free(p, off, bytes);
    return set_error(LBM_ECUDA, std::string("admitting an instance: ") + cudaGetErrorString(e));
  }
  Slot& sl = p->slots[s];
  std::memset(sl.desc, 0, sizeof(sl.desc));
  if (p->prec == kF64) make_slot_desc<double>(I, steps, reinterpret_cast<PoolSlot<double>*>(sl.desc));
  else make_slot_desc<float>(I, steps, reinterpret_cast<PoolSlot<float>*>(sl.desc));
  sl.desc_pending = true;
  sl.used = true;
  sl.ticket = p->next_ticket++;
  sl.off = off;
  sl.bytes = bytes;
  sl.inst = I;
  sl.steps_total = steps;
  sl.steps_done = 0;
  p->ticket_slot[sl.ticket] = s;
  p->used_bytes += bytes;
  p->ntiles_host += nt;
  p->tiles_dirty = true;
  *ticket = sl.ticket;
  return LBM_OK;
}

int lbm_pool_run(lbm_pool_handle p, int bundles) {
  if (!p) return set_error(LBM_EINVAL, "pool is NULL");
  if (bundles < 0) return set_error(LBM_EINVAL, "bundles must be >= 0");
  for (int b = 0; b < bundles; ++b) {
    bool pending = false;
    for (const Slot& sl : p->slots) pending = pending || (sl.used && sl.desc_pending);
    if (pending) {
      // the admissions' initialisation precedes the bundle; the descriptors
      // are written between bundles, on the pool stream
      cudaError_t e = cudaStreamWaitEvent(p->stream, p->io_done, 0);
      for (int s = 0; s < p->max_slots && e == cudaSuccess; ++s) {
        Slot& sl = p->slots[s];
        if (!sl.used || !sl.desc_pending) continue;
        e = cudaMemcpyAsync(p->d_slots + (size_t)s * p->slot_size, sl.desc, p->slot_size, cudaMemcpyHostToDevice,
                            p->stream);
        sl.desc_pending = false;
      }
      if (e != cudaSuccess)
        return set_error(LBM_ECUDA, std::string("writing slot descriptors: ") + cudaGetErrorString(e));
      p->tiles_dirty = true;  // upload_tiles synchronises the pool stream: the descriptor sources stay valid
    }
    if (p->tiles_dirty) {
      int rc = upload_tiles(p);
      if (rc != LBM_OK) return rc;
    }
    cudaError_t e = cudaGraphLaunch(p->exec, p->stream);
    if (e != cudaSuccess) return set_error(LBM_ECUDA, std::string("launching a step bundle: ") + cudaGetErrorString(e));
    for (Slot& sl : p->slots)
      if (sl.used) sl.steps_done = std::min(sl.steps_total, sl.steps_done + (long)p->bundle_steps);
  }
  return LBM_OK;
}

int lbm_pool_sync(lbm_pool_handle p) {
  if (!p) return set_error(LBM_EINVAL, "pool is NULL");
  cudaError_t e = cudaStreamSynchronize(p->stream);
  // error words: an instance that met a non-finite state has stopped stepping
  p->h_flags.resize(p->max_slots);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->h_flags.data(), p->d_flags, sizeof(unsigned int) * p->max_slots, cudaMemcpyDeviceToHost,
                        p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return set_error(LBM_ECUDA, std::string("synchronising the pool: ") + cudaGetErrorString(e));
  for (int s = 0; s < p->max_slots; ++s) {
    Slot& sl = p->slots[s];
    if (sl.used && !sl.nonfinite && (p->h_flags[s] & 1u)) {
      sl.nonfinite = true;
      sl.steps_done = sl.steps_total;
    }
  }
  return LBM_OK;
}

int lbm_pool_poll(lbm_pool_handle p, long long ticket, int* done, long* steps_done) {
  if (!p) return set_error(LBM_EINVAL, "pool is NULL");
  auto it = p->ticket_slot.find(ticket);
  if (it == p->ticket_slot.end()) return set_error(LBM_EINVAL, "unknown ticket");
  const Slot& sl = p->slots[it->second];
  if (steps_done) *steps_done = sl.steps_done;
  if (done) *done = sl.steps_done >= sl.steps_total ? 1 : 0;
  return LBM_OK;
}

int lbm_pool_result(lbm_pool_handle p, long long ticket, double* rho, double* u, double* T) {
  if (!p) return set_error(LBM_EINVAL, "pool is NULL");
  auto it = p->ticket_slot.find(ticket);
  if (it == p->ticket_slot.end()) return set_error(LBM_EINVAL, "unknown ticket");
  const int s = it->second;
  Slot& sl = p->slots[s];
  if (sl.steps_done < sl.steps_total) return set_error(LBM_EBUSY, "the instance has steps left");
  Instance& I = sl.inst;
  if (I.N > 0 && (!rho || !u || !T)) return set_error(LBM_EINVAL, "field pointer is NULL");
  if (sl.nonfinite) {
    // stopped early: its fields are not defined; report NaN
    const double nan = std::nan("");
    for (long long k = 0; k < I.N; ++k) rho[k] = T[k] = nan;
    for (long long k = 0; k < I.D * I.N; ++k) u[k] = nan;
    arena_free(p, sl.off, sl.bytes);
    p->used_bytes -= sl.bytes;
    p->ntiles_host -= tiles_of(p, I);
    p->ticket_slot.erase(it);
    sl = Slot();
    p->tiles_dirty = true;
    return set_error(LBM_ENONFINITE, "the instance met a non-finite density or temperature");
  }
  const int cur = (int)(sl.steps_total & 1);
  unsigned int flag = 0;
  cudaError_t e = cudaSuccess;
  if (I.N > 0) {
    double* st = static_cast<double*>(I.buf[cur ^ 1]);
    const size_t nb = sizeof(double) * (size_t)I.N;
    e = p->L->moments(&I, I.buf[cur], st, st + I.N, st + (1 + I.D) * I.N);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rho, st, nb, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(u, st + I.N, nb * I.D, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(T, st + (1 + I.D) * I.N, nb, cudaMemcpyDeviceToHost, p->stream);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, p->d_flags + s, sizeof(flag), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return set_error(LBM_ECUDA, std::string("reading a result: ") + cudaGetErrorString(e));
  // retire: the slot's descriptor already has no steps left; free its memory
  arena_free(p, sl.off, sl.bytes);
  p->used_bytes -= sl.bytes;
  p->ntiles_host -= tiles_of(p, I);
  p->ticket_slot.erase(it);
  sl = Slot();
  p->tiles_dirty = true;
  if (flag & 1u) return set_error(LBM_ENONFINITE, "the instance met a non-finite density or temperature");
  return LBM_OK;
}

int lbm_pool_stats(lbm_pool_handle p, long long* out) {
  if (!p || !out) return set_error(LBM_EINVAL, "NULL argument");
  long long resident = 0, finished = 0;
  for (const Slot& sl : p->slots)
    if (sl.used) {
      ++resident;
      if (sl.steps_done >= sl.steps_total) ++finished;
    }
  out[0] = resident;
  out[1] = finished;
  out[2] = (long long)p->used_bytes;
  out[3] = (long long)p->arena_bytes;
  out[4] = p->ntiles_host;
  out[5] = p->grid;
  return LBM_OK;
}

}  // extern "C"
