// Fused dual-space H application of the FP32 inner CG (Sec. 4.1: kinetic term on the sphere,
// V_loc through the G -> r -> G transforms): the three passes of the pruned FFT pipeline
// (plane g2r, x-line with V(r), plane r2g) run in one kernel with the pair intermediate
// T[h][y][z] held in shared memory instead of HBM.
//
// One thread-block cluster of R CTAs per pair.  The 2m+1 h-planes of the pair are distributed
// over the cluster by plane group {+a, -a} (a = |h|, group a on rank a mod R), so that the r -> G
// unpack of Z(G) and Z(-G) stays inside one CTA.  Stage 1 transforms each CTA's planes along
// z then y in place; stage 2 runs the x-lines (y, z) of its share of the plane, reading and
// writing the 2m+1 values of each line in the planes of every CTA of the cluster through
// distributed shared memory; stage 3 transforms its planes back along y then z in place,
// gathers the sphere, unpacks the pair and applies the epilogue.  Cluster barriers separate the
// stages.  The butterflies are those of the three separate kernels (same radix plans, same
// order; the compiler's FMA contraction differs, so results agree to FP32 rounding); per pair
// the HBM traffic drops from four passes over (2m+1) N^2 complex values to the two sphere
// vectors in and the one out.
#include <cooperative_groups.h>

#include "internal.h"

namespace cg = cooperative_groups;

namespace wgw {
namespace fused {

constexpr int kMaxRanks = 8;
constexpr int kMaxPlanes = 64;

// Where plane hi lives: CTA rank and slot in that CTA's plane buffer; the planes of each rank.
struct PlaneMap {
  signed char rank[kMaxPlanes];
  signed char slot[kMaxPlanes];
  signed char nloc[kMaxRanks];
  signed char hloc[kMaxRanks][kMaxPlanes];
};

template <int N>
struct Tw {
  cplx<float> w[N];
};

template <int N>
constexpr int threads_for() { return N == 48 ? 288 : (N == 32 ? 256 : 192); }

// Pair q is idle when none of its systems is active (the same rule as the separate kernels).
__device__ __forceinline__ bool pair_idle(const int* active, const int* list, int pair, int n_list) {
  int s0, s1;
  pair_members(list, n_list, pair, s0, s1);
  if (s0 < 0) return true;   // past the count of a device-compacted list
  if (active == nullptr) return false;
  return !active[s0] && (s1 < 0 || !active[s1]);
}

template <int N>
__global__ void __launch_bounds__(threads_for<N>(), 1)
k_hpsi_fused(SphereTab sp, const __grid_constant__ Tw<N> tw, const __grid_constant__ PlaneMap pm, const float* P,
             long ldp, int n_list, const int* list, const int* active, const float* V, Epi<float> e) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ cplx<float>* plane_at[kMaxPlanes];   // plane hi in the cluster's shared memory
  cg::cluster_group cluster = cg::this_cluster();
  const int R = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int pair = blockIdx.x / R;
  // Every CTA of the cluster takes the same decision, so none waits at a barrier alone.
  if (pair_idle(active, list, pair, n_list)) return;
  constexpr int LS = N + 1, NT = threads_for<N>();
  const int m = sp.m, NR = 2 * m + 1;
  const int tid = threadIdx.x;
  cplx<float>* Pl = reinterpret_cast<cplx<float>*>(smem_raw);   // plane q at Pl + q N LS, [row][col]
  const int nloc = pm.nloc[rank];
  int s0, s1;
  pair_members(list, n_list, pair, s0, s1);
  const bool has1 = s1 >= 0;

  // ---- stage 1: G -> r along z (rows |k| <= m), then along y (columns), in place.
  for (int i = tid; i < nloc * NR * LS; i += NT) {
    const int q = i / (NR * LS), r = i % (NR * LS);
    Pl[(size_t)q * N * LS + r] = mk<float>(0.f, 0.f);
  }
  __syncthreads();
  {
    const float* x0 = P + (size_t)s0 * ldp;
    const float* x1 = P + (size_t)(has1 ? s1 : s0) * ldp;
    const float s = kInvSqrt2;
    for (int q = 0; q < nloc; ++q) {
      const int hi = pm.hloc[rank][q];
      cplx<float>* Bq = Pl + (size_t)q * N * LS;
      for (int en_i = sp.plane_off[hi] + tid; en_i < sp.plane_off[hi + 1]; en_i += NT) {
        const int2 en = sp.ent[en_i];
        const int kk = en.x & 0xff, ll = (en.x >> 8) & 0xff, neg = (en.x >> 16) & 1;
        const int kr = kk <= m ? kk + m : kk - N + m;
        const int j = en.y;
        cplx<float> z;
        if (j == 0) {
          z = mk<float>(x0[0], has1 ? x1[0] : 0.f);
        } else {
          const float ar = x0[2 * j - 1], ai = x0[2 * j];
          const float br = has1 ? x1[2 * j - 1] : 0.f, bi = has1 ? x1[2 * j] : 0.f;
          z = neg ? mk<float>((ar + bi) * s, (br - ai) * s) : mk<float>((ar - bi) * s, (ai + br) * s);
        }
        Bq[kr * LS + ll] = z;
      }
    }
  }
  __syncthreads();
  for (int t = tid; t < nloc * NR; t += NT) {          // rows: l -> z
    const int q = t / NR, kr = t % NR;
    cplx<float>* row = Pl + (size_t)q * N * LS + (size_t)kr * LS;
    cplx<float> v[N];
#pragma unroll
    for (int x = 0; x < N; ++x) v[x] = row[x];
    reg_dif<float, N, 0, +1>(v, tw.w);
#pragma unroll
    for (int x = 0; x < N; ++x) row[x] = v[x];
  }
  __syncthreads();
  for (int t = tid; t < nloc * N; t += NT) {           // columns: k -> y, written over the column
    const int q = t / N, zc = t % N;
    cplx<float>* Bq = Pl + (size_t)q * N * LS;
    cplx<float> v[N];
#pragma unroll
    for (int y = 0; y < N; ++y) {
      const int kr = y <= m ? y + m : (y >= N - m ? y - N + m : -1);
      v[y] = kr >= 0 ? Bq[kr * LS + zc] : mk<float>(0.f, 0.f);
    }
    reg_dif<float, N, 0, +1>(v, tw.w);
#pragma unroll
    for (int y = 0; y < N; ++y) Bq[y * LS + zc] = v[y];
  }
  for (int hi = tid; hi < NR; hi += NT)
    plane_at[hi] = cluster.map_shared_rank(Pl, (unsigned)pm.rank[hi]) + (size_t)pm.slot[hi] * N * LS;
  cluster.sync();

  // ---- stage 2: x-lines (y, z) of this rank's share: G -> r, times V(r), r -> G.
  {
    const int per = (N * N + R - 1) / R;
    const int l0 = rank * per, l1 = min(N * N, l0 + per);
    for (int l = l0 + tid; l < l1; l += NT) {
      const int y = l / N, z = l % N;
      const size_t off = (size_t)y * LS + z;
      cplx<float> v[N];
#pragma unroll
      for (int x = 0; x < N; ++x) {
        const bool in = x <= m || x >= N - m;
        const int hi = x <= m ? x + m : x - N + m;
        v[x] = in ? plane_at[hi][off] : mk<float>(0.f, 0.f);
      }
      reg_dif<float, N, 0, +1>(v, tw.w);
      const float* vr = V + (size_t)y * N * N + z;
#pragma unroll
      for (int x = 0; x < N; ++x) v[x] = cscale(v[x], vr[(size_t)x * N]);
      reg_dit<float, N, cplan(N).nst - 1, -1>(v, tw.w);
#pragma unroll
      for (int x = 0; x < N; ++x) {
        const bool in = x <= m || x >= N - m;
        const int hi = x <= m ? x + m : x - N + m;
        if (in) plane_at[hi][off] = v[x];
      }
    }
  }
  cluster.sync();   // every remote access of stage 2 is done before any CTA moves on or exits

  // ---- stage 3: r -> G along y (columns, rows |k| <= m kept) then z (rows), in place; gather,
  // unpack the pair and the epilogue per plane group.
  for (int t = tid; t < nloc * N; t += NT) {
    const int q = t / N, zc = t % N;
    cplx<float>* Bq = Pl + (size_t)q * N * LS;
    cplx<float> v[N];
#pragma unroll
    for (int y = 0; y < N; ++y) v[y] = Bq[y * LS + zc];
    reg_dit<float, N, cplan(N).nst - 1, -1>(v, tw.w);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if (k <= m) Bq[(k + m) * LS + zc] = v[k];
      else if (k >= N - m) Bq[(k - N + m) * LS + zc] = v[k];
    }
  }
  __syncthreads();
  for (int t = tid; t < nloc * NR; t += NT) {
    const int q = t / NR, kr = t % NR;
    cplx<float>* row = Pl + (size_t)q * N * LS + (size_t)kr * LS;
    cplx<float> v[N];
#pragma unroll
    for (int x = 0; x < N; ++x) v[x] = row[x];
    reg_dit<float, N, cplan(N).nst - 1, -1>(v, tw.w);
#pragma unroll
    for (int x = 0; x < N; ++x) row[x] = v[x];
  }
  __syncthreads();
  const bool act0 = is_active(e.active, s0), act1 = has1 && is_active(e.active, s1);
  const float scale = (float)(1.0 / ((double)N * N * N));
  for (int q = 0; q < nloc; ++q) {
    const int hi = pm.hloc[rank][q];
    if (hi < m) continue;                 // the group is handled from its +a plane
    const int hp = hi - m;
    const cplx<float>* Bp = Pl + (size_t)q * N * LS;
    const int off_p = sp.plane_off[hi];
    const int cnt = sp.plane_off[hi + 1] - off_p;
    if (hp == 0) {
      const int K = (cnt - 1) / 2;
      for (int t = tid; t < K; t += NT) {
        const int2 ep_ = sp.ent[off_p + 1 + t];
        unpack_store(e, sp, s0, s1, act0, act1, ep_.y, Bp[ent_pos_rows<N>(ep_, m)],
                     Bp[ent_pos_rows<N>(sp.ent[off_p + 1 + K + t], m)], scale);
      }
      if (tid == 0) {
        const cplx<float> z0 = Bp[ent_pos_rows<N>(sp.ent[off_p], m)];
        if (act0) epi_store(e, sp, s0, 0, z0.re * scale);
        if (act1) epi_store(e, sp, s1, 0, z0.im * scale);
      }
      continue;
    }
    const cplx<float>* Bm = Pl + (size_t)pm.slot[m - hp] * N * LS;
    const int off_m = sp.plane_off[m - hp];
    for (int t = tid; t < cnt; t += NT)
      unpack_store(e, sp, s0, s1, act0, act1, sp.ent[off_p + t].y, Bp[ent_pos_rows<N>(sp.ent[off_p + t], m)],
                   Bm[ent_pos_rows<N>(sp.ent[off_m + t], m)], scale);
  }
}

// The plane groups {+a, -a} dealt to the ranks (a mod R), and the smallest cluster (1, 2, 4, 8)
// whose largest share fits the shared memory of one CTA.
bool plan_map(int N, int m, PlaneMap& pm, int& R, size_t& smem) {
  const size_t plane_bytes = sizeof(cplx<float>) * (size_t)N * (N + 1);
  const size_t limit = 227 * 1024;
  for (R = 1; R <= kMaxRanks; R *= 2) {
    int most = 0;
    for (int r = 0; r < R; ++r) {
      int c = 0;
      for (int a = r; a <= m; a += R) c += a == 0 ? 1 : 2;
      most = std::max(most, c);
    }
    if ((size_t)most * plane_bytes <= limit) break;
  }
  if (R > kMaxRanks || 2 * m + 1 > kMaxPlanes) return false;
  for (int r = 0; r < kMaxRanks; ++r) pm.nloc[r] = 0;
  for (int a = 0; a <= m; ++a) {
    const int r = a % R;
    const int his[2] = {m + a, m - a};
    for (int k = 0; k < (a == 0 ? 1 : 2); ++k) {
      pm.rank[his[k]] = (signed char)r;
      pm.slot[his[k]] = pm.nloc[r];
      pm.hloc[r][(int)pm.nloc[r]] = (signed char)his[k];
      pm.nloc[r] = (signed char)(pm.nloc[r] + 1);
    }
  }
  int most = 0;
  for (int r = 0; r < R; ++r) most = std::max(most, (int)pm.nloc[r]);
  smem = (size_t)most * plane_bytes;
  return true;
}

template <int N>
Tw<N> host_tw() {
  Tw<N> t;
  for (int k = 0; k < N; ++k) {
    const double ang = 2.0 * 3.14159265358979323846 * k / N;
    t.w[k] = mk<float>((float)std::cos(ang), (float)std::sin(ang));
  }
  return t;
}

template <int N>
cudaError_t launch_n(const SphereTab& sp, const float* P, long ldp, int n_list, const int* list, const int* active,
                     const float* V, const Epi<float>& e, cudaStream_t st) {
  static const Tw<N> tw = host_tw<N>();
  PlaneMap pm{};
  int R = 1;
  size_t smem = 0;
  if (!plan_map(N, sp.m, pm, R, smem)) return cudaErrorNotSupported;
  cudaError_t err = ensure_smem_limit((const void*)k_hpsi_fused<N>, smem);
  if (err != cudaSuccess) return err;
  if (R > 1) {
    err = cudaFuncSetAttribute(k_hpsi_fused<N>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (err != cudaSuccess) return err;
  }
  const int pairs = (n_list + 1) / 2;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(pairs * R);
  cfg.blockDim = dim3(threads_for<N>());
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = R;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_hpsi_fused<N>, sp, tw, pm, P, ldp, n_list, list, active, V, e);
}

}  // namespace fused

bool hpsi_fused_supported(int N, int m) {
  if (N != 24 && N != 32 && N != 48) return false;
  fused::PlaneMap pm{};
  int R = 1;
  size_t smem = 0;
  return fused::plan_map(N, m, pm, R, smem);
}

cudaError_t launch_hpsi_fused(const SphereTab& sp, int N, const float* P, long ldp, int n_list, const int* list,
                              const int* active, const float* V, const Epi<float>& e, cudaStream_t st) {
  if (n_list <= 0) return cudaSuccess;
  switch (N) {
    case 24: return fused::launch_n<24>(sp, P, ldp, n_list, list, active, V, e, st);
    case 32: return fused::launch_n<32>(sp, P, ldp, n_list, list, active, V, e, st);
    case 48: return fused::launch_n<48>(sp, P, ldp, n_list, list, active, V, e, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace wgw
