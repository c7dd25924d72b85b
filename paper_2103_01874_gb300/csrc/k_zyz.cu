// Fused spectral middle pass of the direct Poisson solve of Eq. (34) (the fast
// Poisson solver stated after Eq. (34): DFT in the periodic x and z, a
// Neumann solve in y), for power-of-two ny and nz in [32, 256].
//
// Spectrum layout on this path ("plane layout"): complex FP32 [kx][kz][j], j
// fastest, i.e. index kx * (ny nz) + line with line = k ny + j the physical
// x-line; the forward x pass writes it so and the inverse x pass reads it so.
//
// One thread-block cluster of C CTAs owns one kx plane (nz x ny values, 512 KB
// at 256^2), spread over its CTAs' shared memory: CTA r holds the j columns
// [r JC, (r+1) JC) of every kz row, loaded by one bulk tensor copy (TMA)
// whose completion is counted on an mbarrier.  The plane then goes through
//   1. the forward DFT along z of the CTA's JC columns (register-staged passes,
//      in place on the tile);
//   2. a cluster barrier;
//   3. the y solve of the CTA's RC rows kz in [r RC, (r+1) RC): DCT-II of each
//      row (Makhoul's reordering and one complex FFT), division by the
//      eigenvalue lam_x(kx) + lam_y(ky) + lam_z(kz) of the 7-point operator with
//      the zero mode pinned, DCT-III back.  A row's values are read from, and
//      written back to, the tiles of all C CTAs through distributed shared
//      memory; between passes the row sits in a local scratch row;
//   4. a cluster barrier;
//   5. the inverse DFT along z of the CTA's columns;
//   6. one bulk tensor store of the tile.
// So the half spectrum crosses HBM once in and once out for the three steps
// that the separate z, y and z passes each read and wrote in full.  The
// arithmetic is that of k_zfft_rg, k_ydct_rg and k_zfft_rg.
//
// Waits: the tile load is awaited with a bounded number of mbarrier rounds;
// if they run out the CTA records PPE error bit 1 in DevScalars::dev_err,
// still takes part in both cluster barriers (so no CTA of the cluster waits
// forever), skips its compute and its store, and waits once more (bounded)
// for the load before it exits.  No multicast: each copy moves data between
// global memory and one CTA's own shared memory.
#include "ppe_internal.h"
#include "stencil.cuh"
#include "tma.cuh"

namespace ppe {

template <int NY, int NZ>
struct ZyzCfg {
  static constexpr int C = (NY * NZ >= 8192) ? NY * NZ / 8192 : 1;  // CTAs per plane: 64 KB tiles
  static constexpr int JC = NY / C;                                  // j columns per CTA
  static constexpr int RC = NZ / C;                                  // kz rows per CTA in the y step
  static constexpr int THREADS = NY * NZ / (16 * C);                 // 16 elements per thread per step
  // scratch row stride (complex elements): rgfft rows, padded to 8 mod 16
  static constexpr int LSY = rgfft::rows(NY) + ((8 - rgfft::rows(NY) % 16) + 16) % 16;
  static constexpr size_t TILE = (size_t)NZ * JC * 8;
  static constexpr size_t SCR = (size_t)RC * LSY * 8;
  static constexpr size_t TABLES = (size_t)(NZ + 2 * NY) * 8 + (size_t)(NY + NZ) * 4 + 16;
  static constexpr size_t SMEM = 1024 + TILE + SCR + TABLES;  // + alignment slack of the tile
  static_assert(C <= 8, "portable cluster size");
  static_assert(JC % 2 == 0 && JC <= 256 && NZ <= 256, "bulk tensor box");
  static_assert(THREADS % 32 == 0 && THREADS <= 1024, "whole warps");
};

constexpr uint32_t kTmaWaitRounds = 1u << 20;

template <int NY, int NZ>
__global__ void __launch_bounds__(ZyzCfg<NY, NZ>::THREADS, 1)
    k_zyz(GridDev g, const __grid_constant__ CUtensorMap tmap, const cpx<float>* __restrict__ tw_z,
          const cpx<float>* __restrict__ tw_y, const cpx<float>* __restrict__ wq, const float* __restrict__ lam_x,
          const float* __restrict__ lam_y, const float* __restrict__ lam_z, DevScalars* err, DevScalars* fin) {
  using Cfg = ZyzCfg<NY, NZ>;
  using T = float;
  constexpr int C = Cfg::C, JC = Cfg::JC, RC = Cfg::RC, LSY = Cfg::LSY, THREADS = Cfg::THREADS;
  extern __shared__ unsigned char smem_raw[];
  // the tile at a 1024-byte boundary (bulk tensor copies want an aligned base)
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  cpx<T>* tile = reinterpret_cast<cpx<T>*>(base);  // [NZ][JC]
  cpx<T>* scr = tile + NZ * JC;                    // [RC][LSY]
  cpx<T>* tz = scr + RC * LSY;                     // exp(-2 pi i t/nz)
  cpx<T>* ty = tz + NZ;                            // exp(-2 pi i t/ny)
  cpx<T>* wqs = ty + NY;                           // exp(-i pi k/(2 ny))
  T* ly = reinterpret_cast<T*>(wqs + NY);          // lam_y
  T* lz = ly + NY;                                 // lam_z
  uint64_t* bar = reinterpret_cast<uint64_t*>(lz + NZ);

  const int tid = threadIdx.x;
  const uint32_t rank = cluster_ctarank();
  const int kx = (int)(blockIdx.x / C);
  if (fin && blockIdx.x == 0) finish_sums(fin, g);  // uniform over the CTA
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(bar, (uint32_t)Cfg::TILE);
    tma_load_2d(tile, &tmap, bar, (int)rank * JC, kx * NZ);
  }
  for (int t = tid; t < NZ; t += THREADS) {
    tz[t] = tw_z[t];
    lz[t] = lam_z[t];
  }
  for (int t = tid; t < NY; t += THREADS) {
    ty[t] = tw_y[t];
    wqs[t] = wq[t];
    ly[t] = lam_y[t];
  }
  const T lxk = lam_x[kx];
  const bool got = mbar_wait_bounded(bar, 0, kTmaWaitRounds);
  const bool ok = __syncthreads_and(got) != 0;  // uniform over the CTA; also publishes the tables
  if (!ok && tid == 0) atomicOr(&err->dev_err, 1);

  // 1. forward DFT along z of the CTA's columns (column l, thread rank t0 in it)
  const int zl = tid % JC, zt0 = tid / JC;
  cpx<T>* col = tile + zl;
  auto ldc = [&](int e) { return col[e * JC]; };
  auto stc = [&](int e, cpx<T> v) { col[e * JC] = v; };
  if (ok) rgfft::run<T, false, NZ, 1, true, rgfft::DENSE>(ldc, stc, col, JC, zt0, tz);
  cluster_sync();  // 2.

  // 3. y solve of rows kz = rank RC + yl
  {
    constexpr int TP = NY / 16;
    const int yl = tid / TP, yt0 = tid % TP;
    const int kz = (int)rank * RC + yl;
    const uint32_t tile_u = smem_u32(tile);
    cpx<T>* ln = scr + yl * LSY;
    // element p of the reordered row: v[p] = x_j, j = 2p (p < NY/2) or 2(NY-1-p)+1,
    // held by CTA j / JC at (kz, j mod JC)
    auto raddr = [&](int p) -> uint32_t {
      const int j = p < NY / 2 ? 2 * p : 2 * (NY - 1 - p) + 1;
      const int r = j / JC, jl = j - r * JC;
      return mapa(tile_u + (uint32_t)(kz * JC + jl) * 8u, (uint32_t)r);
    };
    if (ok)
      rgfft::run<T, false, NY, 1, false, rgfft::PAD_ROWS>(
          [&](int p) {
            const float2 v = ld_cluster_f2(raddr(p));
            return cpx<T>{v.x, v.y};
          },
          [&](int e, cpx<T> v) { ln[rgfft::row(e)] = v; }, ln, 1, yt0, ty);
    __syncthreads();
    // divide by the eigenvalues (zero mode pinned), combining the DCT-II pair
    // (k, NY-k): X_k = (w_k V_k + conj(w_k) V_{N-k})/2, P = X/lam,
    // V'_k = conj(w_k)(P_k - i P_{N-k})
    constexpr int NP = NY / 2 + 1;
    const T inv_n = (T)1 / (T)NY;
    for (int idx = tid; idx < RC * NP; idx += THREADS) {
      const int rr = idx / NP, k = idx - rr * NP;
      const int kzr = (int)rank * RC + rr;
      const T lxz = lxk + lz[kzr];
      cpx<T>* V = scr + rr * LSY;
      if (k == 0) {
        const cpx<T> v0 = V[0];
        // inv_n / lam as inv_n * (1/lam): inv_n is a power of two
        if (kx == 0 && kzr == 0) {  // zero mode pinned (to the value that keeps p zero-mean)
          V[0] = {(T)err->zmode, (T)0};
          continue;
        }
        const T s = inv_n * __frcp_rn(lxz + ly[0]);
        V[0] = {v0.x * s, v0.y * s};
        continue;
      }
      const int r = NY - k;
      cpx<T>* Vk = V + rgfft::row(k);
      cpx<T>* Vr = V + rgfft::row(r);
      const cpx<T> vk = *Vk, vr = *Vr;
      const cpx<T> wk = wqs[k], wr = wqs[r];
      const cpx<T> wkc = {wk.x, -wk.y}, wrc = {wr.x, -wr.y};
      const cpx<T> t1 = cmul(wk, vk), t2c = cmul(wkc, vr);
      const cpx<T> xk = {(T)0.5 * (t1.x + t2c.x), (T)0.5 * (t1.y + t2c.y)};
      const cpx<T> t3 = cmul(wr, vr), t4 = cmul(wrc, vk);
      const cpx<T> xr = {(T)0.5 * (t3.x + t4.x), (T)0.5 * (t3.y + t4.y)};
      const T sk = inv_n * __frcp_rn(lxz + ly[k]), sr = inv_n * __frcp_rn(lxz + ly[r]);
      const cpx<T> pk = {xk.x * sk, xk.y * sk}, pr = {xr.x * sr, xr.y * sr};
      // -i z = (z.y, -z.x)
      *Vk = cmul(wkc, cpx<T>{pk.x + pr.y, pk.y - pr.x});
      if (r != k) *Vr = cmul(wrc, cpx<T>{pr.x + pk.y, pr.y - pk.x});
    }
    __syncthreads();
    if (ok)
      rgfft::run<T, true, NY, 1, true, rgfft::PAD_ROWS>(
          [&](int e) { return ln[rgfft::row(e)]; },
          [&](int p, cpx<T> v) { st_cluster_f2(raddr(p), make_float2(v.x, v.y)); }, ln, 1, yt0, ty);
  }
  cluster_sync();  // 4. every row is back in every tile; no remote access after this

  // 5. inverse DFT along z, 6. store
  if (ok) rgfft::run<T, true, NZ, 1, true, rgfft::DENSE>(ldc, stc, col, JC, zt0, tz);
  fence_proxy_async_smem();
  __syncthreads();
  if (tid == 0) {
    if (ok) {
      tma_store_2d(&tmap, tile, (int)rank * JC, kx * NZ);
      bulk_commit();
      bulk_wait_all();
    } else {
      mbar_wait_bounded(bar, 0, kTmaWaitRounds);  // a late load must land before the CTA leaves
    }
  }
}

namespace {
template <int NY, int NZ>
cudaError_t go_zyz(const GridDev& g, const CUtensorMap& tmap, const cpx<float>* tw_z, const cpx<float>* tw_y,
                   const cpx<float>* wq, const float* lam_x, const float* lam_y, const float* lam_z, DevScalars* err,
                   DevScalars* fin, cudaStream_t st, int* max_clusters) {
  using Cfg = ZyzCfg<NY, NZ>;
  auto kern = k_zyz<NY, NZ>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
  if (e != cudaSuccess) return e;
  const int nxh = g.nx / 2 + 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(Cfg::C * nxh), 1, 1);
  cfg.blockDim = dim3(Cfg::THREADS, 1, 1);
  cfg.dynamicSmemBytes = Cfg::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = Cfg::C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (max_clusters) return cudaOccupancyMaxActiveClusters(max_clusters, kern, &cfg);
  return cudaLaunchKernelEx(&cfg, kern, g, tmap, tw_z, tw_y, wq, lam_x, lam_y, lam_z, err, fin);
}

template <typename F>
cudaError_t with_ny_nz(int ny, int nz, F&& f) {
  auto by_nz = [&](auto NYC) -> cudaError_t {
    constexpr int NY = decltype(NYC)::value;
    switch (nz) {
      case 32: return f(NYC, std::integral_constant<int, 32>{});
      case 64: return f(NYC, std::integral_constant<int, 64>{});
      case 128: return f(NYC, std::integral_constant<int, 128>{});
      case 256: return f(NYC, std::integral_constant<int, 256>{});
      default: return cudaErrorInvalidValue;
    }
    (void)NY;
  };
  switch (ny) {
    case 32: return by_nz(std::integral_constant<int, 32>{});
    case 64: return by_nz(std::integral_constant<int, 64>{});
    case 128: return by_nz(std::integral_constant<int, 128>{});
    case 256: return by_nz(std::integral_constant<int, 256>{});
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

bool zyz_supported(int ny, int nz) {
  auto ok = [](int n) { return n == 32 || n == 64 || n == 128 || n == 256; };
  return ok(ny) && ok(nz);
}

int zyz_cols(int ny, int nz) {
  int c = 0;
  with_ny_nz(ny, nz, [&](auto A, auto B) -> cudaError_t {
    c = ZyzCfg<decltype(A)::value, decltype(B)::value>::JC;
    return cudaSuccess;
  });
  return c;
}

cudaError_t zyz_max_clusters(const GridDev& g, int* n) {
  *n = 0;
  CUtensorMap dummy = {};
  return with_ny_nz(g.ny, g.nz, [&](auto A, auto B) {
    return go_zyz<decltype(A)::value, decltype(B)::value>(g, dummy, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                          nullptr, nullptr, nullptr, nullptr, n);
  });
}

cudaError_t launch_zyz(const GridDev& g, const CUtensorMap& tmap, const cpx<float>* tw_z, const cpx<float>* tw_y,
                       const cpx<float>* wq, const float* lam_x, const float* lam_y, const float* lam_z,
                       DevScalars* err, DevScalars* fin, cudaStream_t st) {
  return with_ny_nz(g.ny, g.nz, [&](auto A, auto B) {
    return go_zyz<decltype(A)::value, decltype(B)::value>(g, tmap, tw_z, tw_y, wq, lam_x, lam_y, lam_z, err, fin, st,
                                                          nullptr);
  });
}

}  // namespace ppe
