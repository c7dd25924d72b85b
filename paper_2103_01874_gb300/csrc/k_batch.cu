// Persistent batched projection: the FP32 solve + pair refinement form of
// ppe_project (Eqs. (32)-(34) and the fast solve stated after Eq. (34)) for many
// grids of different sizes in ONE launch.
//
// Work queue.  The host lists every (grid, stage, tile) item of the batch in a
// queue order (batch_schedule); each resident CTA repeatedly takes the next
// item (one atomic on the queue head), waits until the grid's previous stage
// has all its tiles done (a per-grid, per-stage device counter), runs the tile
// with the same device function the stage's own kernel uses (one tile = one
// CTA of that kernel), and counts the tile done.  A wait only ever targets an
// item earlier in the queue, taken by a CTA that is already running, so the
// queue cannot deadlock; nevertheless every wait is bounded in time: when one
// runs out, the kernel records PPE_ERR_TIMEOUT (and the grid and stage) in its
// control block and in every grid's dev_err, every CTA stops taking items and
// the launch ends.
//
// Memory ordering.  A tile's writes are ordered before its counter increment by
// __syncthreads and a device-scope fence in the counting thread; the waiting
// thread reads the counter with an acquire load and fences before the CTA
// barrier, so the CTA's loads that follow see the previous stage's data.  The
// buffers the kernel writes are never read through the non-coherent path.
//
// Refinement.  The first launch's queue holds the whole projection with one
// refinement sweep.  A loop test (refine_decide, as the graph form's test
// kernel) that stops its grid marks it stopped; one that asks for another
// sweep sets the control block's cont_any, and the batch graph's WHILE node
// then launches the kernel again over the sweep stages' queue, in which the
// items of stopped grids are skipped.
//
// Items are runs of consecutive tiles of one stage of one grid (about `grain`
// elements), so that the fixed cost of taking, waiting for and counting an
// item is spread over several tiles.
#include <stdio.h>

#include <algorithm>
#include <climits>
#include <type_traits>
#include <vector>

#include "../../include/ppe.h"
#include "correct.cuh"
#include "ppe_internal.h"
#include "rhs.cuh"
#include "spectral.cuh"

namespace ppe {

// ---------------------------------------------------------------------------
// host side: lengths, tiles, queue order
// ---------------------------------------------------------------------------
namespace {
bool len_ok(int n) {
  switch (n) {
    case 32: case 48: case 64: case 96: case 128: case 192: case 256: return true;
    default: return false;
  }
}
bool pow2(int n) { return (n & (n - 1)) == 0; }
unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }
}  // namespace

bool batch_dims_ok(int nx, int ny, int nz) { return len_ok(nx) && len_ok(ny) && len_ok(nz); }

// x passes of a radix-3 nx/2: as many lines as keep the tile within 4096 reals
// (at most 64), as the graph form's default
int batch_lpb(int nx) {
  int l = 1;
  while (2 * l <= 4096 / nx && 2 * l <= 64) l *= 2;
  return l;
}
// z (16) and y (8) columns of a radix-3 length, fewer when the tile would not fit
int batch_tkx(int n, bool zpass) {
  int t = zpass ? 16 : 8;
  while (t > 2 && 8 * (2 * (size_t)t * n + n) > 160 * 1024) t /= 2;
  return t;
}

namespace {
// tiles of a transform pass along a length-n direction: power-of-two lengths
// run the register-staged form with 4096 / n lines (256 threads); radix-3
// lengths the shared-memory form with `cols` lines
unsigned lines_per_tile(int n, int cols) { return pow2(n) ? 4096u / (unsigned)n : (unsigned)cols; }
constexpr size_t kRhoCellsPerTile = 65536;     // rho_0 reduction: 256 threads x 256 cells
constexpr size_t kFacesPerThreadCC = 16;        // correction check: v faces per thread
constexpr int kBatchRhsLines = 1;               // right-hand side: lines per thread stack (registers: no spills)
}  // namespace

unsigned batch_stage_tiles(int nx, int ny, int nz, bool rho_given, int stage) {
  const size_t n = (size_t)nx * ny * nz;
  const int nxh = nx / 2 + 1;
  const unsigned nlines = (unsigned)ny * nz;
  const unsigned x_tiles = cdiv(nlines, lines_per_tile(nx / 2, batch_lpb(nx)));
  const unsigned z_tiles = (unsigned)ny * cdiv(nxh, lines_per_tile(nz, batch_tkx(nz, true)));
  const unsigned y_tiles = (unsigned)nz * cdiv(nxh, lines_per_tile(ny, batch_tkx(ny, false)));
  switch (stage) {
    case BS_RHO: return rho_given ? 0u : cdiv(n, kRhoCellsPerTile);
    case BS_CONST: return 1u;
    case BS_RHS: {
      const int tj = (kRhsThreads / nx) * kBatchRhsLines;
      return cdiv(ny, tj) * cdiv(nz, nz < 8 ? nz : 8);
    }
    case BS_XF: case BS_XI0: case BS_RES: case BS_XA: return x_tiles;
    case BS_ZF0: case BS_ZI0: case BS_ZF: case BS_ZI: return z_tiles;
    case BS_Y0: case BS_Y: return y_tiles;
    case BS_CC: return cdiv((size_t)nz * (ny + 1) * nx, kFacesPerThreadCC * kBatchThreads);
    case BS_CHK: return 1u;
    default: return 0u;
  }
}

unsigned batch_stage_chunk(int nx, int ny, int nz, int stage, long grain) {
  if (grain < 1) grain = 1;
  const long nxh = nx / 2 + 1;
  long per = 1;  // elements of one tile
  switch (stage) {
    case BS_RHO: return 1u;
    case BS_CONST: case BS_CHK: return 1u;
    case BS_RHS: per = (long)(kRhsThreads / nx) * kBatchRhsLines * nx * (nz < 8 ? nz : 8); break;
    case BS_XF: case BS_XI0: case BS_RES: case BS_XA:
      per = (long)lines_per_tile(nx / 2, batch_lpb(nx)) * nx;
      break;
    case BS_ZF0: case BS_ZI0: case BS_ZF: case BS_ZI:
      per = std::min<long>(lines_per_tile(nz, batch_tkx(nz, true)), nxh) * nz;
      break;
    case BS_Y0: case BS_Y: per = std::min<long>(lines_per_tile(ny, batch_tkx(ny, false)), nxh) * ny; break;
    case BS_CC: per = (long)kFacesPerThreadCC * kBatchThreads; break;
    default: return 1u;
  }
  const long c = grain / per;
  return (unsigned)std::max(1L, std::min(255L, c));
}

size_t batch_smem(int nx, int ny, int nz) {
  size_t m = rhs_smem(nx, kBatchRhsLines);
  const int lx = (int)lines_per_tile(nx / 2, batch_lpb(nx));
  m = std::max(m, pow2(nx / 2) ? xrg_smem(nx, lx) : xfwd_smem<float>(nx, lx));
  m = std::max(m, pow2(nx / 2) ? xrg_smem(nx, lx) : xinv_smem<float>(nx, lx));
  m = std::max(m, pow2(nz) ? rg_smem<float>(nz, 4096 / nz) : zfft_smem<float>(nz, batch_tkx(nz, true)));
  m = std::max(m, pow2(ny) ? rg_smem<float>(ny, 4096 / ny) : zfft_smem<float>(ny, batch_tkx(ny, false)));
  return m;
}

long long batch_item_count(int n, const int* nx, const int* ny, const int* nz, const int* rho_given, int first,
                           long grain) {
  long long c = 0;
  for (int g = 0; g < n; ++g)
    for (int s = first; s < kBatchStages; ++s)
      c += cdiv(batch_stage_tiles(nx[g], ny[g], nz[g], rho_given[g] != 0, s),
                batch_stage_chunk(nx[g], ny[g], nz[g], s, grain));
  return c;
}

// Queue order: stage-major within windows of `window` grids (every grid of a
// window has its stage s listed before any of its stage s + 1), window w
// entering `stagger` stages after window w - 1, so that several windows'
// stages are in flight at once while each window's spectra stay few enough to
// be reused from L2.  Ties: larger grids first, then grid index, then tile.  A
// grid's stages keep their order, so every item's dependency is listed before
// it.  need and tiles are
// filled for every stage (also those before `first`).
void batch_schedule(int n, const int* nx, const int* ny, const int* nz, const int* rho_given, int window,
                    int stagger, int first, long grain, BatchItem* items, unsigned* need, unsigned* tiles) {
  if (window < 1) window = 1;
  if (stagger < 0) stagger = 0;
  std::vector<unsigned> chunk((size_t)kBatchStages * n);
  for (int g = 0; g < n; ++g)
    for (int s = 0; s < kBatchStages; ++s) {
      const int i = kBatchStages * g + s;
      tiles[i] = batch_stage_tiles(nx[g], ny[g], nz[g], rho_given[g] != 0, s);
      chunk[i] = batch_stage_chunk(nx[g], ny[g], nz[g], s, grain);
      need[i] = cdiv(tiles[i], chunk[i]);
    }
  struct Key {
    long long k;
    int g, s;
  };
  std::vector<Key> keys;
  for (int g = 0; g < n; ++g)
    for (int s = first; s < kBatchStages; ++s) keys.push_back({(long long)s + (long long)stagger * (g / window), g, s});
  // within a key, larger grids first: their longer chains of stages start
  // earlier (then grid index, stage)
  auto cells = [&](int g) { return (double)nx[g] * ny[g] * nz[g]; };
  std::stable_sort(keys.begin(), keys.end(), [&](const Key& a, const Key& b) {
    if (a.k != b.k) return a.k < b.k;
    if (cells(a.g) != cells(b.g)) return cells(a.g) > cells(b.g);
    return a.g != b.g ? a.g < b.g : a.s < b.s;
  });
  size_t m = 0;
  for (const Key& k : keys) {
    const int i = kBatchStages * k.g + k.s;
    for (unsigned t = 0; t < tiles[i]; t += chunk[i])
      items[m++] = {(uint16_t)k.g, (uint8_t)k.s, (uint8_t)std::min(chunk[i], tiles[i] - t), t};
  }
}

// ---------------------------------------------------------------------------
// device side
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// f(std::integral_constant<int, M>) for the x half-lengths M = nx / 2
template <typename F>
__device__ __forceinline__ void on_xhalf(int m, F&& f) {
  switch (m) {
    case 16: f(std::integral_constant<int, 16>{}); break;
    case 24: f(std::integral_constant<int, 24>{}); break;
    case 32: f(std::integral_constant<int, 32>{}); break;
    case 48: f(std::integral_constant<int, 48>{}); break;
    case 64: f(std::integral_constant<int, 64>{}); break;
    case 96: f(std::integral_constant<int, 96>{}); break;
    case 128: f(std::integral_constant<int, 128>{}); break;
    default: break;
  }
}
// the same for the z and y lengths
template <typename F>
__device__ __forceinline__ void on_len(int n, F&& f) {
  switch (n) {
    case 32: f(std::integral_constant<int, 32>{}); break;
    case 48: f(std::integral_constant<int, 48>{}); break;
    case 64: f(std::integral_constant<int, 64>{}); break;
    case 96: f(std::integral_constant<int, 96>{}); break;
    case 128: f(std::integral_constant<int, 128>{}); break;
    case 192: f(std::integral_constant<int, 192>{}); break;
    case 256: f(std::integral_constant<int, 256>{}); break;
    default: break;
  }
}

// forward x pass of f (SRC_FDF) or of the residual (SRC_RESID), tile t of nt
template <int SRC>
__device__ __noinline__ void x_forward(const BatchGrid* __restrict__ Bp, uint32_t t, uint32_t nt) {
  const BatchGrid& B = *Bp;
  on_xhalf(B.g.nx / 2, [&](auto MC) {
    constexpr int M = decltype(MC)::value;
    if constexpr (rgfft::is_rg<M>::value) {
      xfwd_rg_body<SRC, M, false, false>(B.g, B.in, B.sc, SRC == SRC_RESID ? -1 : 0, B.fdf, B.pdf, B.spec, B.tw_x,
                                         4096 / M, t, nt);
    } else {
      RadixPlan rp;  // (compile-time lengths: the radix plan is not read)
      xfwd_body<float, SRC, true, M, false>(B.g, B.in, B.sc, SRC == SRC_RESID ? -1 : 0, B.fdf, B.pdf, B.spec, rp,
                                            B.tw_x, B.lpb, t, nt);
    }
  });
}

// inverse x pass into the pairs (XI_DF) or added to them (XI_DF_ACC), with the
// partial sums of p that keep it zero-mean
template <int MODE>
__device__ __noinline__ void x_inverse(const BatchGrid* __restrict__ Bp, uint32_t t, uint32_t nt) {
  const BatchGrid& B = *Bp;
  on_xhalf(B.g.nx / 2, [&](auto MC) {
    constexpr int M = decltype(MC)::value;
    if constexpr (rgfft::is_rg<M>::value) {
      xinv_rg_body<MODE, M, false>(B.g, B.spec, nullptr, B.pdf, B.scale, B.tw_x, 4096 / M, nullptr, B.sc, t, nt);
    } else {
      RadixPlan rp;  // (compile-time lengths: the radix plan is not read)
      xinv_body<float, MODE, M>(B.g, B.spec, nullptr, B.pdf, B.scale, rp, B.tw_x, B.lpb, nullptr, B.sc, t, nt);
    }
  });
}

// z pass; the forward one totals the partial sums first in its tile 0 (fin)
template <bool INV>
__device__ __noinline__ void z_pass(const BatchGrid* __restrict__ Bp, uint32_t t, uint32_t nt) {
  const BatchGrid& B = *Bp;
  DevScalars* fin = INV ? nullptr : B.sc;
  on_len(B.g.nz, [&](auto NC) {
    constexpr int N = decltype(NC)::value;
    if constexpr (rgfft::is_rg<N>::value) {
      zfft_rg_body<float, INV, N>(B.g, B.spec, B.tw_z, 4096 / N, nullptr, fin, t, nt);
    } else {
      RadixPlan rp;  // (compile-time lengths: the radix plan is not read)
      zfft_body<float, INV, N>(B.g, B.spec, rp, B.tw_z, B.tkx, nullptr, fin, t, nt);
    }
  });
}

// y pass: DCT-II, eigenvalue divide (zero mode from zmode), DCT-III
__device__ __noinline__ void y_pass(const BatchGrid* __restrict__ Bp, uint32_t t, uint32_t nt) {
  const BatchGrid& B = *Bp;
  on_len(B.g.ny, [&](auto NC) {
    constexpr int N = decltype(NC)::value;
    if constexpr (N == 256) {  // the radix-16 x 16 form with the divide in registers, as the graph form
      ydct256_body(B.g, B.spec, B.tw_y, B.wq_y, B.lam_x, B.lam_y, B.lam_z, 16, B.sc, t, nt);
    } else if constexpr (rgfft::is_rg<N>::value) {
      ydct_rg_body<float, N>(B.g, B.spec, B.tw_y, B.wq_y, B.lam_x, B.lam_y, B.lam_z, 4096 / N, B.sc, t, nt);
    } else {
      RadixPlan rp;  // (compile-time lengths: the radix plan is not read)
      ydct_body<float, N>(B.g, B.spec, rp, B.tw_y, B.wq_y, B.lam_x, B.lam_y, B.lam_z, B.tky, B.sc, t, nt);
    }
  });
}

__device__ __noinline__ void rhs_pass(const BatchGrid* __restrict__ Bp, uint32_t t) {
  const BatchGrid& B = *Bp;
  RhsOut o;
  o.f64 = B.f64;
  o.fdf = B.fdf;
  o.upre = B.upre;
  o.vpre = B.vpre;
  o.wpre = B.wpre;
  if (B.in.face_rule == 0) rhs_stack_tile<kBatchRhsLines, 0, true>(B.g, B.in, B.sc, o, B.kc, t);
  else rhs_stack_tile<kBatchRhsLines, 1, true>(B.g, B.in, B.sc, o, B.kc, t);
}

__device__ __noinline__ void rho_pass(const BatchGrid* __restrict__ Bp, uint32_t t, uint32_t nt) {
  rho_min_body(Bp->in.rho, (size_t)Bp->g.nx * Bp->g.ny * Bp->g.nz, Bp->sc, t, nt);
}

__device__ __noinline__ void cc_pass(const BatchGrid* __restrict__ Bp, uint32_t t, uint32_t nt) {
  const BatchGrid& B = *Bp;
  correct_check_tile(B.g, B.upre, B.vpre, B.wpre, B.pdf, B.fdf, B.sc, t, nt);
}

// Runs tile t of stage s of grid B (nt tiles in the stage); returns, for the
// loop test, whether the refinement goes on (1) or stops (0); -1 otherwise.
__device__ __forceinline__ int run_item(const BatchGrid* __restrict__ Bp, int s, uint32_t t, uint32_t nt) {
  switch (s) {
    case BS_RHO: rho_pass(Bp, t, nt); break;
    case BS_CONST:
      if (threadIdx.x == 0) Bp->sc->K = make_const(Bp->g, read_rho0(Bp->sc), Bp->in.dt);
      break;
    case BS_RHS: rhs_pass(Bp, t); break;
    case BS_XF: x_forward<SRC_FDF>(Bp, t, nt); break;
    case BS_ZF0: case BS_ZF: z_pass<false>(Bp, t, nt); break;
    case BS_Y0: case BS_Y: y_pass(Bp, t, nt); break;
    case BS_ZI0: case BS_ZI: z_pass<true>(Bp, t, nt); break;
    case BS_XI0: x_inverse<XI_DF>(Bp, t, nt); break;
    case BS_RES: x_forward<SRC_RESID>(Bp, t, nt); break;
    case BS_XA: x_inverse<XI_DF_ACC>(Bp, t, nt); break;
    case BS_CC: cc_pass(Bp, t, nt); break;
    default: return threadIdx.x == 0 ? refine_decide(Bp->sc, Bp->smax, 1) : -1;  // BS_CHK
  }
  return -1;
}

enum WaitResult { W_RUN = 0, W_SKIP = 1, W_ABORT = 2 };

// Thread 0: waits until stage s-1 of grid g has all its tiles done (or, `hold`
// set, on a counter nothing increments: the test of the bounded wait).  The
// sweep stages of a grid whose loop test has stopped it are skipped.  The
// acquire load that ends the wait orders the CTA's later loads (after the CTA
// barrier) after the previous stage's writes.
__device__ int wait_ready(const BatchItem it, const BatchGrid* grids, int ngrid, const unsigned* done,
                          const unsigned* need, const int* stop, BatchCtl* ctl, unsigned long long wait_ns,
                          int hold, int ndone) {
  const int g = it.grid, s = it.stage;
  const bool sweep = s >= BS_RES;
  if (sweep && ld_relaxed_s32(stop + g)) return W_SKIP;
  int dep = -1;
  unsigned target = 0;
  if (hold && g == 0 && s == BS_CONST) {
    dep = ndone;  // the sentinel counter past the stages
    target = 1;
  } else if (s > 0) {
    dep = kBatchStages * g + s - 1;
    target = need[dep];
  }
  if (dep < 0 || ld_acquire_u32(done + dep) >= target) return W_RUN;
  const unsigned long long t0 = global_ns();
  for (;;) {
    __nanosleep(64);
    if (ld_acquire_u32(done + dep) >= target) return W_RUN;
    if (ld_relaxed_s32(&ctl->abort)) return W_ABORT;
    if (global_ns() - t0 > wait_ns) {
      if (atomicCAS(&ctl->status, 0, (int)PPE_ERR_TIMEOUT) == 0) {
        ctl->err_grid = g;
        ctl->err_stage = s;
      }
      for (int i = 0; i < ngrid; ++i) atomicOr(&grids[i].sc->dev_err, 4);
      __threadfence();
      atomicExch(&ctl->abort, 1);
      return W_ABORT;
    }
  }
}

__device__ __forceinline__ void count_done(unsigned* p) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
}

__global__ void __launch_bounds__(kBatchThreads, 3)
    k_batch(const BatchGrid* __restrict__ grids, int ngrid, const BatchItem* __restrict__ items, int nitems,
            unsigned* done, int ndone, const unsigned* __restrict__ need, const unsigned* __restrict__ tiles,
            int* stop, BatchCtl* ctl, unsigned long long wait_ns, int hold) {
  __shared__ int s_item, s_state;
  // thread 0 takes the next item while the current one runs (one item of
  // look-ahead: the smallest unfinished item is always running or runnable)
  unsigned q_next = 0;
  if (threadIdx.x == 0) q_next = atomicAdd(&ctl->next, 1u);
  for (;;) {
    if (threadIdx.x == 0) {
      int it = -1, state = W_ABORT;
      const unsigned q = q_next;
      if (q < (unsigned)nitems && !ld_relaxed_s32(&ctl->abort)) {
        it = (int)q;
        state = wait_ready(items[q], grids, ngrid, done, need, stop, ctl, wait_ns, hold, ndone);
        if (state != W_ABORT) q_next = atomicAdd(&ctl->next, 1u);
      }
      s_item = it;
      s_state = state;
    }
    __syncthreads();
    const int q = s_item, state = s_state;
    if (q < 0 || state == W_ABORT) break;  // uniform over the CTA
    if (state == W_RUN) {
      const BatchItem it = items[q];
      const BatchGrid* B = grids + it.grid;
      const int si = kBatchStages * it.grid + it.stage;
      const unsigned nt = tiles[si];
      for (unsigned t = it.tile0; t < it.tile0 + it.count; ++t) {
        if (t > it.tile0) __syncthreads();  // the previous tile's shared-memory reads
        const int cont = run_item(B, it.stage, t, nt);
        if (threadIdx.x == 0 && cont >= 0) {
          if (cont == 0) stop[it.grid] = 1;
          else ctl->cont_any = 1;
        }
      }
      __syncthreads();  // the item's writes (and its shared-memory reads) before the count
      if (threadIdx.x == 0) count_done(done + si);
    }
    __syncthreads();  // s_item is rewritten by the next take
  }
}

// Per-call state of every grid (as k_init_scalars with the outputs recorded),
// the stage counters, the stop marks and the control block.
__global__ void k_batch_reset(const BatchGrid* __restrict__ grids, int ngrid, unsigned* done, int ndone, int* stop,
                              BatchCtl* ctl) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  for (int i = tid; i <= ndone; i += gridDim.x * blockDim.x) done[i] = 0u;  // (ndone: the sentinel)
  for (int g = tid; g < ngrid; g += gridDim.x * blockDim.x) {
    const BatchGrid& B = grids[g];
    init_scalars(B.sc, B.rho0, B.tol, 0, B.out_p, B.out_u, B.out_v, B.out_w);
    stop[g] = 0;
  }
  if (tid == 0) {
    ctl->next = 0u;
    ctl->abort = 0;
    ctl->status = 0;
    ctl->err_grid = -1;
    ctl->err_stage = -1;
    ctl->cont_any = 0;
    ctl->launches = 1;
  }
}

// Before a further sweep: the sweep stages' counters and the queue head.
__global__ void k_batch_sweep_reset(int ngrid, unsigned* done, BatchCtl* ctl) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int per = kBatchStages - BS_RES;
  for (int i = tid; i < ngrid * per; i += gridDim.x * blockDim.x) done[kBatchStages * (i / per) + BS_RES + i % per] = 0u;
  if (tid == 0) {
    ctl->next = 0u;
    ctl->cont_any = 0;
    ctl->launches += 1;
  }
}

__global__ void k_batch_cond(BatchCtl* ctl, cudaGraphConditionalHandle h) {
  if (threadIdx.x == 0) cudaGraphSetConditional(h, (ctl->cont_any && !ctl->abort) ? 1u : 0u);
}

}  // namespace

cudaError_t batch_occupancy(size_t smem, int* ctas_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_batch, kBatchThreads, smem);
}

cudaError_t launch_batch_reset(const BatchGrid* grids, int ngrid, unsigned* done, int ndone, int* stop,
                               BatchCtl* ctl, cudaStream_t st) {
  const int rb = std::min(std::max(ngrid, ndone + 1) / 256 + 1, 64);
  k_batch_reset<<<rb, 256, 0, st>>>(grids, ngrid, done, ndone, stop, ctl);
  return cudaGetLastError();
}

cudaError_t launch_batch_sweep_reset(const BatchGrid* grids, int ngrid, unsigned* done, BatchCtl* ctl,
                                     cudaStream_t st) {
  (void)grids;
  const int rb = std::min(ngrid * (kBatchStages - BS_RES) / 256 + 1, 64);
  k_batch_sweep_reset<<<rb, 256, 0, st>>>(ngrid, done, ctl);
  return cudaGetLastError();
}

cudaError_t launch_batch(const BatchGrid* grids, int ngrid, const BatchItem* items, int nitems, unsigned* done,
                         int ndone, const unsigned* need, const unsigned* tiles, int* stop, BatchCtl* ctl,
                         unsigned long long wait_ns, int hold, int ctas, size_t smem, cudaStream_t st) {
  if (ngrid < 1 || nitems < 1 || ctas < 1) return cudaErrorInvalidValue;
  k_batch<<<ctas, kBatchThreads, smem, st>>>(grids, ngrid, items, nitems, done, ndone, need, tiles, stop, ctl,
                                             wait_ns, hold);
  return cudaGetLastError();
}

cudaError_t launch_batch_cond(BatchCtl* ctl, cudaGraphConditionalHandle h, cudaStream_t st) {
  k_batch_cond<<<1, 32, 0, st>>>(ctl, h);
  return cudaGetLastError();
}

}  // namespace ppe
