// Transport sweep: local factorisation, dependency-driven wavefront solve, FP64 residual
// and mixed-precision defect correction, and source iteration.
//
// The element equations (upwind DG, pointwise upwinding at face Gauss points) give, for
// direction d and element e,
//     A_{e,d} psi_e = b_e - sum_{inflow faces f} Cin_{f} u_f,
//     A_{e,d} = sigma_t M_e - mu Gx_e - eta Gy_e + sum_f sum_k max(c_k, 0) l_a(s_k) l_b(s_k),
//     (Cin_f)_{a t} = sum_k min(c_k, 0) l_a(s_k) l_t(s_k),   c_k = w_k Omega . (n ds)_k,
// with u_f the upwind neighbour's face-node values (GLL basis: its trace on the shared face
// is spanned by its p+1 face nodes).  Only the u_f terms depend on other elements.
//
// factor_kernel (factor.cu; no dependencies, one thread per (element, direction)) assembles
// A and inverts it in place by Gauss-Jordan elimination, and forms W_f = A^{-1} Cin_f for the
// interior inflow faces.  The record per (element, direction) is
//     [A^{-1} column-major n x n][W_0 ... W_3, each column-major n x (p+1)].
// sweep_kernel then only does, per element, psi = A^{-1} b - sum_f W_f u_f, one lane per
// dof row, so that the chain of dependent work per wavefront level is a few FMAs (on this
// GPU a warp-wide FP64 FMA occupies its SM sub-partition for ~64 cycles, so per-element
// latency, not total flops, bounds a naive wavefront).
//
// Warps claim warp-sized chunks of independent tasks in increasing order from one
// counter; each task waits (bounded) on the completion epochs of its upwind donors,
// which the schedule places in earlier chunks, so the kernel makes progress without any
// assumption on block residency.
#include <algorithm>
#include <cmath>

#include "device.cuh"

namespace vef {


// ----------------------------------------------------------------- right-hand sides
// bvol[e][i] = sum_j M_ij (sigma_s phi_in_j / (4 pi) + q_j)  (isotropic, direction-free)
__global__ void bvol_kernel(long long E, int n, const double* __restrict__ M,
                            const double* __restrict__ sigma_s, const double* __restrict__ phi_in,
                            const double* __restrict__ q, double* __restrict__ bvol) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= E * n) return;
  long long e = t / n;
  int i = (int)(t % n);
  const double ss = phi_in ? sigma_s[e] / kFourPi : 0.0;
  double s = 0.0;
  for (int j = 0; j < n; ++j) {
    double v = 0.0;
    if (phi_in) v += ss * phi_in[e * n + j];
    if (q) v += q[e * n + j];
    s += M[(e * n + i) * n + j] * v;
  }
  bvol[t] = s;
}

// --------------------------------------------------------------------------- sweep
template <typename T>
struct SweepArgs {
  int nchunks;
  const int* chunk_begin;
  const int* slot_first;
  const int* slot_count;
  const uint32_t* code;
  const int* member_of;
  const uint16_t* finfo;
  const double* omega;
  const T* rec;
  const double* bvol;      // [E][n] (mode 0)
  const double* src_aniso; // [D][E][n] or null (mode 0)
  const double* Mm;        // FP64 mass matrices (anisotropic source)
  const double* inflow;    // [D][nbf][nq] or null (mode 0)
  const T* nds;            // [E][4][nq][2]
  const double* rhs;       // [D][E][n] (mode 1)
  T* out;                  // [D][E][n]
  uint32_t* flags;         // [D][E]
  uint32_t epoch;
  unsigned int* status;    // [0] bits, [1] abort, [2] max inner iterations, [3] chunk counter
  int nx, ny;
  long long E, nbf;
  T tol;
  int max_inner;
  FaceTab<T> ft;
};

// own right-hand-side entry b_i of (d, e): volume source plus boundary inflow (mode 0),
// or the given residual (mode 1)
template <int P, typename T, int MODE>
__device__ __forceinline__ T rhs_entry(const SweepArgs<T>& a, int d, int e, int i, uint16_t bits,
                                       T mu, T eta) {
  constexpr int Q = P + 1, N = Q * Q, NQ = P + 2;
  if (MODE == 1) return (T)a.rhs[((size_t)d * a.E + e) * N + i];
  double b = a.bvol[(size_t)e * N + i];
  if (a.src_aniso) {
    const double* Mr = a.Mm + ((size_t)e * N + i) * N;
    const double* qd = a.src_aniso + ((size_t)d * a.E + e) * N;
#pragma unroll
    for (int j = 0; j < N; ++j) b += Mr[j] * qd[j];
  }
  T bt = (T)b;
  if (a.inflow) {
    const int ia = i % Q, ib = i / Q;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      if (!(bits & (1u << f))) continue;
      if (nb_elem(a.nx, a.ny, e, f) >= 0) continue;
      int pos = -1;
      if (f == 0 && ib == 0) pos = ia;
      if (f == 1 && ia == P) pos = ib;
      if (f == 2 && ib == P) pos = ia;
      if (f == 3 && ia == 0) pos = ib;
      if (pos < 0) continue;
      const int bf = bface(a.nx, a.ny, e, f);
      const double* pb = a.inflow + ((size_t)d * a.nbf + bf) * NQ;
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        const T* v = a.nds + (((size_t)e * 4 + f) * NQ + k) * 2;
        const T s = a.ft.w[k] * (mu * v[0] + eta * v[1]);
        if (s < (T)0) bt -= s * (T)pb[k] * a.ft.l[pos][k];
      }
    }
  }
  return bt;
}

template <int P, typename T, int MODE>
__global__ void __launch_bounds__(128) sweep_kernel(SweepArgs<T> a) {
  constexpr int Q = P + 1, N = Q * Q, R = rec_size<P>();
  constexpr int SPC = (32 / N) > 0 ? (32 / N) : 1;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  while (true) {
    int c = 0;
    if (lane == 0) c = (int)atomicAdd(a.status + 3, 1u);
    c = __shfl_sync(FULL, c, 0);
    if (c >= a.nchunks) return;
    if (*((volatile unsigned int*)(a.status + 1)) != 0u) return;
    const int s0 = a.chunk_begin[c], s1 = a.chunk_begin[c + 1];
    const int cnt0 = a.slot_count[s0];
    if (cnt0 == 1) {
      // ---- up to SPC independent single-element tasks, N lanes each
      const int slot = s0 + lane / N;
      const int i = lane % N;
      const bool valid = (lane < SPC * N) && (slot < s1);
      int d = 0, e = 0;
      long long m = 0;
      uint16_t bits = 0;
      T mu = 0, eta = 0;
      T bi = 0;
      if (valid) {
        m = a.slot_first[slot];
        const uint32_t cd = a.code[m];
        d = (int)(cd >> 22);
        e = (int)(cd & 0x3fffffu);
        bits = a.finfo[(size_t)d * a.E + e];
        mu = (T)a.omega[2 * d];
        eta = (T)a.omega[2 * d + 1];
        bi = rhs_entry<P, T, MODE>(a, d, e, i, bits, mu, eta);
      }
      const T* rec = a.rec + (size_t)m * R;
      const int base = (lane / N) * N;
      T y = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const T bj = __shfl_sync(FULL, bi, (base + j) & 31);
        if (valid) y += rec[j * N + i] * bj;
      }
      bool ok = true;
      if (valid) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          if (!(bits & (1u << f))) continue;
          const int nb = nb_elem(a.nx, a.ny, e, f);
          if (nb < 0) continue;
          if (!wait_epoch(a.flags + (size_t)d * a.E + nb, a.epoch, a.status)) { ok = false; break; }
        }
      }
      if (!__all_sync(FULL, ok)) return;
      if (valid) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          if (!(bits & (1u << f))) continue;
          const int nb = nb_elem(a.nx, a.ny, e, f);
          if (nb < 0) continue;
          const T* un = a.out + ((size_t)d * a.E + nb) * N;
          const T* W = rec + N * N + f * N * Q;
#pragma unroll
          for (int t = 0; t < Q; ++t) y -= W[t * N + i] * ldcg(un + face_dof<P>((f + 2) & 3, t));
        }
        a.out[((size_t)d * a.E + e) * N + i] = y;
      }
      __threadfence();
      __syncwarp();
      if (valid && i == 0) st_release(a.flags + (size_t)d * a.E + e, a.epoch);
    } else {
      // ---- one strongly coupled group: members in order, block Gauss-Seidel to tol
      const int first = a.slot_first[s0];
      const int cnt = cnt0;
      const int i = lane;
      const bool act = lane < N;
      const uint32_t c0 = a.code[first];
      const int d = (int)(c0 >> 22);
      const T mu = (T)a.omega[2 * d], eta = (T)a.omega[2 * d + 1];
      bool ok = true;
      // wait on every external donor first
      for (int mi = 0; mi < cnt && ok; ++mi) {
        const int e = (int)(a.code[first + mi] & 0x3fffffu);
        const uint16_t bits = a.finfo[(size_t)d * a.E + e];
        for (int f = 0; f < 4; ++f) {
          if (!(bits & (1u << f)) || (bits & (1u << (4 + f)))) continue;
          const int nb = nb_elem(a.nx, a.ny, e, f);
          if (nb < 0) continue;
          if (!wait_epoch(a.flags + (size_t)d * a.E + nb, a.epoch, a.status)) { ok = false; break; }
        }
      }
      if (!__all_sync(FULL, ok)) return;
      int it = 0;
      bool conv = false;
      for (; it < a.max_inner; ++it) {
        T dmax = 0, amax = 0;
        for (int mi = 0; mi < cnt; ++mi) {
          const long long m = first + mi;
          const int e = (int)(a.code[m] & 0x3fffffu);
          const uint16_t bits = a.finfo[(size_t)d * a.E + e];
          const T* rec = a.rec + (size_t)m * R;
          T bi = act ? rhs_entry<P, T, MODE>(a, d, e, i, bits, mu, eta) : (T)0;
          T y = 0;
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const T bj = __shfl_sync(FULL, bi, j & 31);
            if (act) y += rec[j * N + i] * bj;
          }
          if (act) {
            for (int f = 0; f < 4; ++f) {
              if (!(bits & (1u << f))) continue;
              const int nb = nb_elem(a.nx, a.ny, e, f);
              if (nb < 0) continue;
              if ((bits & (1u << (4 + f))) && it == 0) {
                const int pos = a.member_of[(size_t)d * a.E + nb] - first;
                if (pos >= mi) continue;  // not computed yet in the first sweep
              }
              const T* un = a.out + ((size_t)d * a.E + nb) * N;
              const T* W = rec + N * N + f * N * Q;
#pragma unroll
              for (int t = 0; t < Q; ++t) y -= W[t * N + i] * ldcg(un + face_dof<P>((f + 2) & 3, t));
            }
            T* o = a.out + ((size_t)d * a.E + e) * N + i;
            if (it > 0) dmax = fmax(dmax, fabs(y - ldcg(o)));
            amax = fmax(amax, fabs(y));
            *o = y;
          }
          __threadfence();
          __syncwarp();
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          dmax = fmax(dmax, __shfl_xor_sync(FULL, dmax, off));
          amax = fmax(amax, __shfl_xor_sync(FULL, amax, off));
        }
        if (it > 0 && dmax <= a.tol * amax) { conv = true; ++it; break; }
      }
      if (lane == 0) {
        if (!conv) atomicOr(a.status, kDevNotConverged);
        atomicMax(a.status + 2, (unsigned)it);
      }
      __threadfence();
      __syncwarp();
      for (int mi = lane; mi < cnt; mi += 32) {
        const int e = (int)(a.code[first + mi] & 0x3fffffu);
        st_release(a.flags + (size_t)d * a.E + e, a.epoch);
      }
    }
  }
}

// -------------------------------------------------------------- FP64 residual (mixed)
// r = b - L psi for all (d, e), one lane per dof row; accumulates ||r||^2, ||b||^2.
template <int P>
__global__ void __launch_bounds__(128)
residual_kernel(int D, long long E, int nx, int ny, long long nbf, const double* __restrict__ omega,
                const double* __restrict__ sigma_t, const double* __restrict__ Mm,
                const double* __restrict__ Gxm, const double* __restrict__ Gym,
                const double* __restrict__ nds, const double* __restrict__ bvol,
                const double* __restrict__ src_aniso, const double* __restrict__ inflow,
                const double* __restrict__ psi, FaceTab<double> ft, double* __restrict__ r,
                double* __restrict__ norms) {
  constexpr int Q = P + 1, N = Q * Q, NQ = P + 2;
  constexpr int SPC = (32 / N) > 0 ? (32 / N) : 1;
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long task = warp * SPC + lane / N;
  const int i = lane % N;
  double rr = 0.0, bb = 0.0;
  if (lane < SPC * N && task < (long long)D * E) {
    const int d = (int)(task / E);
    const int e = (int)(task % E);
    const double mu = omega[2 * d], eta = omega[2 * d + 1], st = sigma_t[e];
    const double* pe = psi + ((size_t)d * E + e) * N;
    double b = bvol[(size_t)e * N + i];
    const double* Mr = Mm + ((size_t)e * N + i) * N;
    const double* Xr = Gxm + ((size_t)e * N + i) * N;
    const double* Yr = Gym + ((size_t)e * N + i) * N;
    if (src_aniso) {
      const double* qd = src_aniso + ((size_t)d * E + e) * N;
      for (int j = 0; j < N; ++j) b += Mr[j] * qd[j];
    }
    double Apsi = 0.0;
#pragma unroll
    for (int j = 0; j < N; ++j) Apsi += (st * Mr[j] - mu * Xr[j] - eta * Yr[j]) * pe[j];
    const int ia = i % Q, ib = i / Q;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      int pos = -1;
      if (f == 0 && ib == 0) pos = ia;
      if (f == 1 && ia == P) pos = ib;
      if (f == 2 && ib == P) pos = ia;
      if (f == 3 && ia == 0) pos = ib;
      if (pos < 0) continue;
      const int nb = nb_elem(nx, ny, e, f);
      const double* pn = nb >= 0 ? psi + ((size_t)d * E + nb) * N : nullptr;
      const double* pb = (nb < 0 && inflow) ? inflow + ((size_t)d * nbf + bface(nx, ny, e, f)) * NQ : nullptr;
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        const double* v = nds + (((size_t)e * 4 + f) * NQ + k) * 2;
        const double s = ft.w[k] * (mu * v[0] + eta * v[1]);
        if (s >= 0.0) {
          double tr = 0.0;
#pragma unroll
          for (int t = 0; t < Q; ++t) tr += ft.l[t][k] * pe[face_dof<P>(f, t)];
          Apsi += s * tr * ft.l[pos][k];
        } else if (pn) {
          double tr = 0.0;
#pragma unroll
          for (int t = 0; t < Q; ++t) tr += ft.l[t][k] * pn[face_dof<P>((f + 2) & 3, t)];
          Apsi += s * tr * ft.l[pos][k];  // upwind coupling belongs to L psi
        } else if (pb) {
          b -= s * pb[k] * ft.l[pos][k];
        }
      }
    }
    const double ri = b - Apsi;
    r[((size_t)d * E + e) * N + i] = ri;
    rr = ri * ri;
    bb = b * b;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, off);
    bb += __shfl_xor_sync(0xffffffffu, bb, off);
  }
  if (lane == 0 && (rr != 0.0 || bb != 0.0)) {
    atomicAdd(norms, rr);
    atomicAdd(norms + 1, bb);
  }
}

__global__ void cast_add_kernel(long long n, const float* __restrict__ delta, double* __restrict__ psi,
                                int accumulate) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  psi[t] = accumulate ? psi[t] + (double)delta[t] : (double)delta[t];
}

// phi[e][i] = sum_d w_d psi[d][e][i]
__global__ void phi_kernel(int D, long long En, const double* __restrict__ w,
                           const double* __restrict__ psi, double* __restrict__ phi) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= En) return;
  double s = 0.0;
  for (int d = 0; d < D; ++d) s += w[d] * psi[(size_t)d * En + t];
  phi[t] = s;
}

// out = max |a - b| (non-negative doubles order like their bit patterns)
__global__ void maxdiff_kernel(long long n, const double* __restrict__ a, const double* __restrict__ b,
                               unsigned long long* out) {
  double m = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(a[t] - (b ? b[t] : 0.0)));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// ------------------------------------------------------------------------ host side
static inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <typename K>
static int persistent_blocks(K kernel, int threads) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0);
  return std::max(1, sms * std::max(1, per));
}

struct SweepCall {
  Mesh* mesh;
  Schedule* S;
  const double* sigma_t;
  const double* sigma_s;
  const double* src_aniso;
  const double* inflow;
  cudaStream_t stream;
  double tol;
  int max_passes;
  int precision;
  int threads;
};

template <int P, typename T, int MODE>
static vef_status launch_sweep(const SweepCall& c, const double* rhs, T* out) {
  Mesh& M = *c.mesh;
  Schedule& S = *c.S;
  SweepArgs<T> a{};
  a.nchunks = S.nchunks;
  a.chunk_begin = S.chunk_begin;
  a.slot_first = S.slot_first;
  a.slot_count = S.slot_count;
  a.code = S.member_code;
  a.member_of = S.member_of;
  a.finfo = S.faceinfo;
  a.omega = S.omega_dev;
  a.rec = (const T*)(std::is_same<T, double>::value ? S.rec64 : S.rec32);
  a.bvol = M.bvol;
  a.src_aniso = c.src_aniso;
  a.Mm = M.Mmat;
  a.inflow = c.inflow;
  a.nds = (const T*)(std::is_same<T, double>::value ? (const void*)M.nds : (const void*)M.nds32);
  a.rhs = rhs;
  a.out = out;
  a.flags = M.flags;
  if (++M.epoch == 0) {
    VEF_CUDA_TRY(cudaMemsetAsync(M.flags, 0, M.flags_cap, c.stream));
    M.epoch = 1;
  }
  a.epoch = M.epoch;
  a.status = M.dev_status;
  a.nx = M.nx;
  a.ny = M.ny;
  a.E = M.E;
  a.nbf = M.nbf;
  const double eps = std::is_same<T, double>::value ? 2.2e-16 : 1.2e-7;
  a.tol = (T)std::max(c.tol, 8.0 * eps);
  a.max_inner = std::max(2, 4 * c.max_passes);
  a.ft = make_facetab<T>(M.tab);
  // reset abort word and chunk counter (status bits [0] and max-inner [2] accumulate
  // until the next synchronising call)
  VEF_CUDA_TRY(cudaMemsetAsync(M.dev_status + 1, 0, sizeof(unsigned int), c.stream));
  VEF_CUDA_TRY(cudaMemsetAsync(M.dev_status + 3, 0, sizeof(unsigned int), c.stream));
  const int threads = c.threads > 0 ? c.threads : 128;
  const int blocks = persistent_blocks(sweep_kernel<P, T, MODE>, threads);
  KTimer kt(&M, VEF_K_SWEEP, c.stream);
  sweep_kernel<P, T, MODE><<<blocks, threads, 0, c.stream>>>(a);
  VEF_CUDA_TRY(cudaGetLastError());
  return VEF_OK;
}

template <int P>
static vef_status launch_residual(const SweepCall& c, const double* psi, double* r, double* norms) {
  Mesh& M = *c.mesh;
  Schedule& S = *c.S;
  constexpr int N = (P + 1) * (P + 1);
  constexpr int SPC = (32 / N) > 0 ? (32 / N) : 1;
  const long long tasks = (long long)S.D * M.E;
  const long long warps = (tasks + SPC - 1) / SPC;
  VEF_CUDA_TRY(cudaMemsetAsync(norms, 0, 2 * sizeof(double), c.stream));
  KTimer kt(&M, VEF_K_RESIDUAL, c.stream);
  residual_kernel<P><<<nblk(warps * 32, 128), 128, 0, c.stream>>>(
      S.D, M.E, M.nx, M.ny, M.nbf, S.omega_dev, c.sigma_t, M.Mmat, M.Gx, M.Gy, M.nds, M.bvol,
      c.src_aniso, c.inflow, psi, make_facetab<double>(M.tab), r, norms);
  VEF_CUDA_TRY(cudaGetLastError());
  return VEF_OK;
}

// One full transport inversion into psi (FP64 output), factors assumed current.
template <int P>
static vef_status solve_p(const SweepCall& c, double* psi, vef_info* info) {
  Mesh& M = *c.mesh;
  Schedule& S = *c.S;
  if (c.precision == VEF_FP64) {
    vef_status st = launch_sweep<P, double, 0>(c, nullptr, psi);
    if (info) { info->passes = 1; info->rel_residual = -1.0; }
    return st;
  }
  // mixed: FP32 sweeps inside FP64 defect correction
  const long long tot = (long long)S.D * M.E * M.n;
  size_t need = (size_t)tot * sizeof(double) + 64;
  vef_status st = ensure_buffer((void**)&M.work2, &M.work2_cap, need + (size_t)tot * sizeof(float));
  if (st != VEF_OK) return st;
  double* r = M.work2;
  double* norms = (double*)((char*)M.work2 + (size_t)tot * sizeof(double));
  float* delta = (float*)((char*)M.work2 + need);
  if ((st = launch_sweep<P, float, 0>(c, nullptr, delta)) != VEF_OK) return st;
  {
    KTimer kt(&M, VEF_K_SOURCE, c.stream);
    cast_add_kernel<<<nblk(tot, 256), 256, 0, c.stream>>>(tot, delta, psi, 0);
  }
  int passes = 1;
  double rel = -1.0;
  for (int pass = 0; pass < c.max_passes; ++pass) {
    if ((st = launch_residual<P>(c, psi, r, norms)) != VEF_OK) return st;
    double h[2];
    VEF_CUDA_TRY(cudaMemcpyAsync(h, norms, sizeof(h), cudaMemcpyDeviceToHost, c.stream));
    VEF_CUDA_TRY(cudaStreamSynchronize(c.stream));
    rel = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
    if (rel <= c.tol) break;
    if (pass == c.max_passes - 1) {
      unsigned int bit = kDevNotConverged;
      VEF_CUDA_TRY(cudaMemcpyAsync(M.dev_status + 4, &bit, sizeof(bit), cudaMemcpyHostToDevice, c.stream));
      break;
    }
    if ((st = launch_sweep<P, float, 1>(c, r, delta)) != VEF_OK) return st;
    {
      KTimer kt(&M, VEF_K_SOURCE, c.stream);
      cast_add_kernel<<<nblk(tot, 256), 256, 0, c.stream>>>(tot, delta, psi, 1);
    }
    ++passes;
  }
  if (info) { info->passes = passes; info->rel_residual = rel; }
  return VEF_OK;
}

static vef_status solve(const SweepCall& c, double* psi, vef_info* info) {
  switch (c.mesh->p) {
    case 1: return solve_p<1>(c, psi, info);
    case 2: return solve_p<2>(c, psi, info);
    case 3: return solve_p<3>(c, psi, info);
    default: return solve_p<4>(c, psi, info);
  }
}

static vef_status factor(const SweepCall& c) {
  return factor_records(c.mesh, c.S, c.sigma_t, c.precision, c.stream);
}

vef_status ensure_flags(Mesh* mesh, size_t count) {
  if (mesh->flags_cap >= count * sizeof(uint32_t)) return VEF_OK;
  vef_status st = ensure_buffer((void**)&mesh->flags, &mesh->flags_cap, count * sizeof(uint32_t));
  if (st != VEF_OK) return st;
  VEF_CUDA_TRY(cudaMemset(mesh->flags, 0, mesh->flags_cap));
  mesh->epoch = 0;
  return VEF_OK;
}

static vef_status launch_bvol(Mesh& M, const double* sigma_s, const double* phi_in,
                              const double* q_iso, cudaStream_t stream) {
  size_t cap = 0;
  if (!M.bvol) {
    vef_status st = ensure_buffer((void**)&M.bvol, &cap, (size_t)M.E * M.n * sizeof(double));
    if (st != VEF_OK) return st;
  }
  KTimer kt(&M, VEF_K_SOURCE, stream);
  bvol_kernel<<<nblk(M.E * M.n, 256), 256, 0, stream>>>(M.E, M.n, M.Mmat, sigma_s, phi_in, q_iso, M.bvol);
  VEF_CUDA_TRY(cudaGetLastError());
  return VEF_OK;
}

// Read back and clear the device status; map to a vef_status.
vef_status collect_status(Mesh& M, cudaStream_t stream, vef_info* info) {
  unsigned int h[8];
  VEF_CUDA_TRY(cudaMemcpyAsync(h, M.dev_status, sizeof(h), cudaMemcpyDeviceToHost, stream));
  VEF_CUDA_TRY(cudaStreamSynchronize(stream));
  unsigned int zero[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  VEF_CUDA_TRY(cudaMemcpyAsync(M.dev_status, zero, sizeof(zero), cudaMemcpyHostToDevice, stream));
  VEF_CUDA_TRY(cudaStreamSynchronize(stream));
  const unsigned bits = h[0] | h[4];
  if (info) {
    info->timed_out = (bits & kDevTimeout) ? 1 : 0;
    info->max_inner_iterations = (int)h[2];
  }
  if (bits & kDevTimeout) { set_last_error("a sweep dependency wait ran out"); return VEF_ERR_TIMEOUT; }
  if (bits & kDevSingular) { set_last_error("singular local element system"); return VEF_ERR_NOT_CONVERGED; }
  if (bits & kDevNotConverged) { set_last_error("an iteration reached its cap"); return VEF_ERR_NOT_CONVERGED; }
  if (bits & kDevNonpositive) { set_last_error("non-positive closure denominator"); return VEF_ERR_NONPOSITIVE_DENOM; }
  return VEF_OK;
}

static vef_status check_common(vef_mesh mesh, const double* omega, const double* weights, int D,
                               const vef_opts* opts) {
  if (!mesh) { set_last_error("mesh is NULL"); return VEF_ERR_INVALID_ARG; }
  if (!omega || !weights) { set_last_error("omega and weights (host arrays) are required"); return VEF_ERR_INVALID_ARG; }
  if (D < 1 || D > kMaxD) { set_last_error("D must be in 1..1023"); return VEF_ERR_INVALID_ARG; }
  for (int d = 0; d < D; ++d) {
    if (!std::isfinite(omega[2 * d]) || !std::isfinite(omega[2 * d + 1]) || !std::isfinite(weights[d])) {
      set_last_error("omega / weights must be finite");
      return VEF_ERR_INVALID_ARG;
    }
  }
  if (opts && opts->precision != VEF_FP64 && opts->precision != VEF_MIXED) {
    set_last_error("opts->precision must be VEF_FP64 or VEF_MIXED");
    return VEF_ERR_INVALID_ARG;
  }
  int dev = 0;
  VEF_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != mesh->impl.device) { set_last_error("mesh belongs to another device"); return VEF_ERR_INVALID_ARG; }
  return VEF_OK;
}

static void fill_opts(const vef_opts* o, SweepCall& c) {
  c.precision = o ? o->precision : VEF_FP64;
  const double deftol = c.precision == VEF_FP64 ? 1e-15 : 1e-13;
  c.tol = (o && o->tol > 0.0) ? o->tol : deftol;
  c.max_passes = (o && o->max_passes > 0) ? o->max_passes : 8;
  c.threads = (o && o->tile_override > 0) ? o->tile_override : 0;
  if (c.threads % 32 != 0 || c.threads > 1024) c.threads = 0;
}

static void schedule_info(const Schedule& S, vef_info* info) {
  if (!info) return;
  info->coupled_groups = S.coupled_groups;
  info->lagged_face_points = S.lagged_points;
  info->levels = S.levels;
}

}  // namespace vef

using namespace vef;

extern "C" vef_status vef_sweep(vef_mesh mesh, const double* sigma_t, const double* sigma_s,
                                const double* phi_in, const double* source, int source_aniso,
                                const double* inflow, const double* omega, const double* weights,
                                int D, const vef_opts* opts, double* psi, vef_info* info,
                                void* stream) {
  vef_status st = check_common(mesh, omega, weights, D, opts);
  if (st != VEF_OK) return st;
  if (!sigma_t || !sigma_s || !psi) { set_last_error("sigma_t, sigma_s and psi are required"); return VEF_ERR_INVALID_ARG; }
  Mesh& M = mesh->impl;
  cudaStream_t s = (cudaStream_t)stream;
  Schedule* S = get_schedule(&M, omega, weights, D, s, &st);
  if (!S) return st;
  if ((st = ensure_flags(&M, (size_t)D * M.E)) != VEF_OK) return st;
  SweepCall c{};
  c.mesh = &M;
  c.S = S;
  c.sigma_t = sigma_t;
  c.sigma_s = sigma_s;
  c.src_aniso = source_aniso ? source : nullptr;
  c.inflow = inflow;
  c.stream = s;
  fill_opts(opts, c);
  if ((st = launch_bvol(M, sigma_s, phi_in, source_aniso ? nullptr : source, s)) != VEF_OK) return st;
  if ((st = factor(c)) != VEF_OK) return st;
  if ((st = solve(c, psi, info)) != VEF_OK) return st;
  if (info) {
    schedule_info(*S, info);
    return collect_status(M, s, info);
  }
  return VEF_OK;
}

extern "C" vef_status vef_source_iterate(vef_mesh mesh, const double* sigma_t, const double* sigma_s,
                                         const double* phi0, const double* source, int source_aniso,
                                         const double* inflow, const double* omega,
                                         const double* weights, int D, int K, const vef_opts* opts,
                                         double* phi_out, double* psi, double* dphi_inf,
                                         vef_info* info, void* stream) {
  vef_status st = check_common(mesh, omega, weights, D, opts);
  if (st != VEF_OK) return st;
  if (!sigma_t || !sigma_s || !psi || !phi_out || K < 1) {
    set_last_error("sigma_t, sigma_s, psi, phi_out are required and K >= 1");
    return VEF_ERR_INVALID_ARG;
  }
  Mesh& M = mesh->impl;
  cudaStream_t s = (cudaStream_t)stream;
  Schedule* S = get_schedule(&M, omega, weights, D, s, &st);
  if (!S) return st;
  if ((st = ensure_flags(&M, (size_t)D * M.E)) != VEF_OK) return st;
  SweepCall c{};
  c.mesh = &M;
  c.S = S;
  c.sigma_t = sigma_t;
  c.sigma_s = sigma_s;
  c.src_aniso = source_aniso ? source : nullptr;
  c.inflow = inflow;
  c.stream = s;
  fill_opts(opts, c);
  const long long En = M.E * M.n;
  if ((st = ensure_buffer((void**)&M.work, &M.work_cap, (size_t)2 * En * sizeof(double))) != VEF_OK)
    return st;
  double* cur = M.work;
  double* nxt = M.work + En;
  if (phi0) VEF_CUDA_TRY(cudaMemcpyAsync(cur, phi0, En * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else VEF_CUDA_TRY(cudaMemsetAsync(cur, 0, En * sizeof(double), s));
  if ((st = factor(c)) != VEF_OK) return st;
  vef_info last{};
  int total_passes = 0;
  for (int k = 0; k < K; ++k) {
    if ((st = launch_bvol(M, sigma_s, cur, source_aniso ? nullptr : source, s)) != VEF_OK) return st;
    if ((st = solve(c, psi, info ? &last : nullptr)) != VEF_OK) return st;
    total_passes += info ? last.passes : 1;
    {
      KTimer kt(&M, VEF_K_SOURCE, s);
      phi_kernel<<<nblk(En, 256), 256, 0, s>>>(D, En, S->weights_dev, psi, nxt);
    }
    if (dphi_inf) {
      VEF_CUDA_TRY(cudaMemsetAsync(dphi_inf + k, 0, sizeof(double), s));
      KTimer kt(&M, VEF_K_SOURCE, s);
      maxdiff_kernel<<<std::min<long long>(nblk(En, 256), 1024), 256, 0, s>>>(
          En, nxt, cur, (unsigned long long*)(dphi_inf + k));
    }
    std::swap(cur, nxt);
  }
  VEF_CUDA_TRY(cudaMemcpyAsync(phi_out, cur, En * sizeof(double), cudaMemcpyDeviceToDevice, s));
  VEF_CUDA_TRY(cudaGetLastError());
  if (info) {
    *info = last;
    info->passes = total_passes;
    schedule_info(*S, info);
    return collect_status(M, s, info);
  }
  return VEF_OK;
}

extern "C" vef_status vef_mesh_sync(vef_mesh mesh, void* stream) {
  if (!mesh) { set_last_error("mesh is NULL"); return VEF_ERR_INVALID_ARG; }
  return collect_status(mesh->impl, (cudaStream_t)stream, nullptr);
}

namespace vef {
vef_status factor_fp64(Mesh* mesh, Schedule* S, const double* sigma_t, cudaStream_t stream) {
  SweepCall c{};
  c.mesh = mesh;
  c.S = S;
  c.sigma_t = sigma_t;
  c.stream = stream;
  c.precision = VEF_FP64;
  c.max_passes = 8;
  c.tol = 1e-15;
  return factor(c);
}
}  // namespace vef
