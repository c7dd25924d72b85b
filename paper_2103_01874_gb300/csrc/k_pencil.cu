// Bulk-copy-staged z and y passes of the direct Poisson solve of Eq. (34) (the
// fast Poisson solver stated after Eq. (34): DFT in the periodic z, a Neumann
// solve in y) on the plane layout of the spectrum, complex FP32 [kx][kz][j]
// with j fastest (index kx * ny nz + kz ny + j).
//
//   k_zfft_tma  DFT along z of a tile of JT j-columns by nz kz-rows of one kx
//               plane (JT nz = 4096 values, 32 KB), moved by 2-D bulk tensor
//               copies (TMA) described by a tensor map of the spectrum.
//   k_ydct_tma  the y solve of a tile of RT consecutive rows (kx, kz), each a
//               contiguous run of ny values (RT ny = 4096, 32 KB), moved by 1-D
//               bulk copies: DCT-II (Makhoul's reordering, one complex FFT),
//               division by the eigenvalue lam_x(kx) + lam_y(ky) + lam_z(kz) of
//               the 7-point operator with the zero mode pinned, DCT-III.
//
// Both are persistent: CTA b walks the tiles b, b + G, b + 2G, ... with two
// shared-memory buffers.  Thread 0 issues the copy of the next tile into the
// other buffer (after the store that last read that buffer has finished
// reading it) before the CTA transforms the current tile in place, then
// stores the current tile; so the loads, the transform and the stores of
// consecutive tiles overlap, and no thread issues a per-element global load
// or store.  Each load is awaited on an mbarrier with a bounded number of
// rounds; if they run out the CTA records bit 1 in DevScalars::dev_err, waits
// (bounded) for the load it left in flight and returns.
//
// The transforms are those of k_zfft_rg and k_ydct_rg (register-staged
// Stockham passes): the z tile is transformed in place column by column
// (dense rows; a warp's lanes are consecutive columns), the y rows in place
// with the intermediate elements at XOR-permuted positions within each row
// (rgfft::XOR_ROWS), so that neither needs padding and the bulk copies see
// dense rows.
#include "ppe_internal.h"
#include "stencil.cuh"
#include "tma.cuh"

namespace ppe {

constexpr uint32_t kPencilWaitRounds = 1u << 20;
constexpr int kPencilTile = 4096;  // complex values per tile (32 KB)

// smem: two tiles, then the tables
template <typename Tab>
__device__ __forceinline__ Tab* after_tiles(unsigned char* base) {
  return reinterpret_cast<Tab*>(base + 2 * kPencilTile * sizeof(cpx<float>));
}

__device__ __forceinline__ unsigned char* aligned_1k(unsigned char* raw) {
  return raw + ((1024u - (smem_u32(raw) & 1023u)) & 1023u);
}

// A load wait of iteration i ran out: record it, then wait once more (bounded)
// for the copies this CTA has in flight -- the tile of iteration i (buffer
// i & 1) and, if issued, the next one (the other buffer) -- so that none lands
// in shared memory after the CTA has left.
__device__ __forceinline__ void pencil_fail(DevScalars* err, uint64_t* bar, int i, bool pref) {
  atomicOr(&err->dev_err, 1);
  mbar_wait_bounded(&bar[i & 1], (uint32_t)(i >> 1) & 1u, kPencilWaitRounds);
  if (pref) mbar_wait_bounded(&bar[(i + 1) & 1], (uint32_t)((i + 1) >> 1) & 1u, kPencilWaitRounds);
}

// DFT along z; NZ in {32, 64, 128, 256}; JT = min(ny, 4096 / NZ) columns per tile;
// tiles: nxh (ny / JT), tile t = (kx = t / (ny/JT), j0 = (t mod (ny/JT)) JT)
template <bool INV, int NZ>
__global__ void __launch_bounds__(256) k_zfft_tma(GridDev g, const __grid_constant__ CUtensorMap tmap,
                                                   const cpx<float>* __restrict__ tw, int jt, DevScalars* err,
                                                   DevScalars* fin) {
  using T = float;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = aligned_1k(smem_raw);
  cpx<T>* buf0 = reinterpret_cast<cpx<T>*>(base);
  cpx<T>* tws = after_tiles<cpx<T>>(base);
  uint64_t* bar = reinterpret_cast<uint64_t*>(tws + NZ);
  const int tid = threadIdx.x;
  if (fin && blockIdx.x == 0) finish_sums(fin, g);  // uniform over the CTA
  const int tpp = g.ny / jt;                          // tiles per kx plane
  const int ntiles = (g.nx / 2 + 1) * tpp;
  const uint32_t bytes = (uint32_t)(jt * NZ) * 8u;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
  }
  for (int t = tid; t < NZ; t += blockDim.x) tws[t] = tw[t];
  __syncthreads();
  auto coords = [&](int t, int& x, int& y) {
    const int kx = t / tpp;
    x = (t - kx * tpp) * jt;
    y = kx * NZ;
  };
  int t = blockIdx.x;
  if (tid == 0 && t < ntiles) {
    int x, y;
    coords(t, x, y);
    mbar_arrive_expect_tx(&bar[0], bytes);
    tma_load_2d(buf0, &tmap, &bar[0], x, y);
  }
  const int l = tid % jt, t0 = tid / jt;  // column, thread rank within it
  bool ok = true;
  int ifail = -1;  // iteration whose load wait ran out
  bool pref = false;  // that iteration had also issued the next tile's load
  for (int i = 0; t < ntiles; t += gridDim.x, ++i) {
    const int b = i & 1;
    cpx<T>* cur = buf0 + b * kPencilTile;
    const int tn = t + gridDim.x;
    if (tid == 0 && tn < ntiles) {
      bulk_wait_read_all();  // the store from the other buffer has read it
      int x, y;
      coords(tn, x, y);
      mbar_arrive_expect_tx(&bar[b ^ 1], bytes);
      tma_load_2d(buf0 + (b ^ 1) * kPencilTile, &tmap, &bar[b ^ 1], x, y);
    }
    ok = __syncthreads_and(mbar_wait_bounded(&bar[b], (uint32_t)(i >> 1) & 1u, kPencilWaitRounds)) != 0;
    if (!ok) {
      ifail = i;
      pref = tn < ntiles;
      break;
    }
    cpx<T>* col = cur + l;
    rgfft::run<T, INV, NZ, 1, true, rgfft::DENSE>([&](int e) { return col[e * jt]; },
                                                  [&](int e, cpx<T> v) { col[e * jt] = v; }, col, jt, t0, tws);
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      int x, y;
      coords(t, x, y);
      tma_store_2d(&tmap, cur, x, y);
      bulk_commit();
    }
  }
  if (tid == 0) {
    if (!ok) pencil_fail(err, bar, ifail, pref);
    bulk_wait_all();
  }
}

// y solve; NY in {32, 64, 128, 256}; RT = 4096 / NY rows per tile; rows r in
// [0, nxh nz), row r = (kx = r / nz, kz = r mod nz); the last tile may be short.
template <int NY>
__global__ void __launch_bounds__(256) k_ydct_tma(GridDev g, cpx<float>* spec, const cpx<float>* __restrict__ tw,
                                                   const cpx<float>* __restrict__ wq,
                                                   const float* __restrict__ lam_x, const float* __restrict__ lam_y,
                                                   const float* __restrict__ lam_z, DevScalars* err) {
  using T = float;
  constexpr int RT = kPencilTile / NY;  // rows per tile
  constexpr int TP = NY / 16;           // threads per row
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = aligned_1k(smem_raw);
  cpx<T>* buf0 = reinterpret_cast<cpx<T>*>(base);
  cpx<T>* tws = after_tiles<cpx<T>>(base);  // exp(-2 pi i t/ny)
  cpx<T>* wqs = tws + NY;                   // exp(-i pi k/(2 ny))
  T* ly = reinterpret_cast<T*>(wqs + NY);
  uint64_t* bar = reinterpret_cast<uint64_t*>(ly + NY);
  const int tid = threadIdx.x;
  const int nz = g.nz, nxh = g.nx / 2 + 1;
  const int nrows = nxh * nz;
  const int ntiles = (nrows + RT - 1) / RT;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
  }
  for (int t = tid; t < NY; t += blockDim.x) {
    tws[t] = tw[t];
    wqs[t] = wq[t];
    ly[t] = lam_y[t];
  }
  __syncthreads();
  auto tile_rows = [&](int t) { return min(RT, nrows - t * RT); };
  auto load = [&](int t, int b) {
    const uint32_t bytes = (uint32_t)(tile_rows(t) * NY) * 8u;
    mbar_arrive_expect_tx(&bar[b], bytes);
    bulk_load_1d(buf0 + b * kPencilTile, spec + (size_t)t * RT * NY, bytes, &bar[b]);
  };
  int t = blockIdx.x;
  if (tid == 0 && t < ntiles) load(t, 0);
  const int ll = tid / TP, t0 = tid % TP;  // row of the tile, thread rank within it
  // v[p] = x_j with j = 2p (p < NY/2) or 2(NY-1-p)+1
  auto jof = [](int p) { return p < NY / 2 ? 2 * p : 2 * (NY - 1 - p) + 1; };
  auto xr = [](int e) { return rgfft::rowp<rgfft::XOR_ROWS>(e); };
  const T inv_n = (T)1 / (T)NY;
  bool ok = true;
  int ifail = -1;
  bool pref = false;
  for (int i = 0; t < ntiles; t += gridDim.x, ++i) {
    const int b = i & 1;
    cpx<T>* cur = buf0 + b * kPencilTile;
    const int tn = t + gridDim.x;
    if (tid == 0 && tn < ntiles) {
      bulk_wait_read_all();
      load(tn, b ^ 1);
    }
    ok = __syncthreads_and(mbar_wait_bounded(&bar[b], (uint32_t)(i >> 1) & 1u, kPencilWaitRounds)) != 0;
    if (!ok) {
      ifail = i;
      pref = tn < ntiles;
      break;
    }
    const int rows = tile_rows(t);
    cpx<T>* ln = cur + ll * NY;
    // forward: DCT-II's FFT of the reordered row, in place (intermediates XOR-permuted)
    rgfft::run<T, false, NY, 1, true, rgfft::XOR_ROWS>([&](int p) { return ln[jof(p)]; },
                                                       [&](int e, cpx<T> v) { ln[xr(e)] = v; }, ln, 1, t0, tws);
    __syncthreads();
    // divide by the eigenvalues (zero mode pinned); pair (k, NY-k) as in k_ydct_rg
    constexpr int NP = NY / 2 + 1;
    for (int idx = tid; idx < rows * NP; idx += blockDim.x) {
      const int rr = idx / NP, k = idx - rr * NP;
      const int r = t * RT + rr;
      const int kx = r / nz, kz = r - kx * nz;
      const T lxz = lam_x[kx] + lam_z[kz];
      cpx<T>* V = cur + rr * NY;
      if (k == 0) {
        const cpx<T> v0 = V[0];
        // inv_n / lam as inv_n * (1/lam): inv_n is a power of two
        if (kx == 0 && kz == 0) {  // zero mode pinned (to the value that keeps p zero-mean)
          V[0] = {(T)err->zmode, (T)0};
          continue;
        }
        const T s = inv_n * __frcp_rn(lxz + ly[0]);
        V[0] = {v0.x * s, v0.y * s};
        continue;
      }
      const int rk = NY - k;
      cpx<T>* Vk = V + xr(k);
      cpx<T>* Vr = V + xr(rk);
      const cpx<T> vk = *Vk, vr = *Vr;
      const cpx<T> wk = wqs[k], wr = wqs[rk];
      const cpx<T> wkc = {wk.x, -wk.y}, wrc = {wr.x, -wr.y};
      const cpx<T> t1 = cmul(wk, vk), t2c = cmul(wkc, vr);
      const cpx<T> xk = {(T)0.5 * (t1.x + t2c.x), (T)0.5 * (t1.y + t2c.y)};
      const cpx<T> t3 = cmul(wr, vr), t4 = cmul(wrc, vk);
      const cpx<T> xrr = {(T)0.5 * (t3.x + t4.x), (T)0.5 * (t3.y + t4.y)};
      const T sk = inv_n * __frcp_rn(lxz + ly[k]), sr = inv_n * __frcp_rn(lxz + ly[rk]);
      const cpx<T> pk = {xk.x * sk, xk.y * sk}, pr = {xrr.x * sr, xrr.y * sr};
      // -i z = (z.y, -z.x)
      *Vk = cmul(wkc, cpx<T>{pk.x + pr.y, pk.y - pr.x});
      if (rk != k) *Vr = cmul(wrc, cpx<T>{pr.x + pk.y, pr.y - pk.x});
    }
    __syncthreads();
    // inverse: DCT-III's FFT, the result back to the reordered positions
    rgfft::run<T, true, NY, 1, true, rgfft::XOR_ROWS>([&](int e) { return ln[xr(e)]; },
                                                      [&](int p, cpx<T> v) { ln[jof(p)] = v; }, ln, 1, t0, tws);
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      bulk_store_1d(spec + (size_t)t * RT * NY, cur, (uint32_t)(rows * NY) * 8u);
      bulk_commit();
    }
  }
  if (tid == 0) {
    if (!ok) pencil_fail(err, bar, ifail, pref);
    bulk_wait_all();
  }
}

namespace {
template <typename K>
int resident_ctas(K kern, int threads, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
}

template <typename F>
cudaError_t with_pow2(int n, F&& f) {
  switch (n) {
    case 32: return f(std::integral_constant<int, 32>{});
    case 64: return f(std::integral_constant<int, 64>{});
    case 128: return f(std::integral_constant<int, 128>{});
    case 256: return f(std::integral_constant<int, 256>{});
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

bool pencil_supported(int ny, int nz) {
  auto ok = [](int n) { return n == 32 || n == 64 || n == 128 || n == 256; };
  return ok(ny) && ok(nz);
}

// j columns of a z tile: 4096 / nz (32 KB tiles), or all ny when fewer
int pencil_zcols(int ny, int nz) { return kPencilTile / nz < ny ? kPencilTile / nz : ny; }

cudaError_t launch_zfft_tma(bool inverse, const GridDev& g, const CUtensorMap& tmap, const cpx<float>* tw,
                            DevScalars* err, DevScalars* fin, cudaStream_t st) {
  return with_pow2(g.nz, [&](auto NC) -> cudaError_t {
    constexpr int NZ = decltype(NC)::value;
    const int jt = pencil_zcols(g.ny, NZ);
    const int threads = jt * NZ / 16;  // 256 (fewer when ny < 4096 / nz)
    const size_t smem = 1024 + 2 * kPencilTile * sizeof(cpx<float>) + NZ * sizeof(cpx<float>) + 16;
    auto go = [&](auto kern) -> cudaError_t {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      static int grid_cap = 0;  // resident CTAs of this instance (per process: one GPU model)
      if (!grid_cap) grid_cap = resident_ctas(kern, threads, smem);
      const int ntiles = (g.nx / 2 + 1) * (g.ny / jt);
      kern<<<ntiles < grid_cap ? ntiles : grid_cap, threads, smem, st>>>(g, tmap, tw, jt, err, fin);
      return cudaGetLastError();
    };
    return inverse ? go(k_zfft_tma<true, NZ>) : go(k_zfft_tma<false, NZ>);
  });
}

cudaError_t launch_ydct_tma(const GridDev& g, cpx<float>* spec, const cpx<float>* tw, const cpx<float>* wq,
                            const float* lam_x, const float* lam_y, const float* lam_z, DevScalars* err,
                            cudaStream_t st) {
  return with_pow2(g.ny, [&](auto NC) -> cudaError_t {
    constexpr int NY = decltype(NC)::value;
    const int threads = kPencilTile / 16;  // RT rows of NY/16 threads: 256
    const size_t smem = 1024 + 2 * kPencilTile * sizeof(cpx<float>) + 2 * NY * sizeof(cpx<float>) +
                        NY * sizeof(float) + 16;
    auto kern = k_ydct_tma<NY>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    static int grid_cap = 0;
    if (!grid_cap) grid_cap = resident_ctas(kern, threads, smem);
    const int rt = kPencilTile / NY;
    const int ntiles = ((g.nx / 2 + 1) * g.nz + rt - 1) / rt;
    kern<<<ntiles < grid_cap ? ntiles : grid_cap, threads, smem, st>>>(g, spec, tw, wq, lam_x, lam_y, lam_z, err);
    return cudaGetLastError();
  });
}

}  // namespace ppe
