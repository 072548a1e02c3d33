// fock_kernels_k.cuh — the Fock apply with Brillouin-zone sampling (§4, the
// E_x equations with sums over k and q and the kernel 1/|G + q|^2), templated
// on the working real type T and the cubic grid size N.
//
// Orbitals are Bloch functions psi_nk = exp(i k.r) u_nk(r); the kernels work on
// the periodic parts u (complex, no symmetry between G and -G).  States are
// numbered s = k * nb + n.  For a pair of states (a, b), q = k_b - k_a and
//   rho_ab = u_a* u_b,   phi_ab = IFFT[v(G + q) FFT(rho_ab)],
//   W_b -= w_a f_a u_a phi_ab,   W_a -= w_b f_b u_b conj(phi_ab)   (a != b)
// (the reverse pair has rho_ba = rho_ab* and q -> -q, so phi_ba = phi_ab*).
// One pair per chain and per complex transform; the whole spectrum is kept.
//
// Layout in HBM:
//   u    [Ns][N][N][N] complex T     periodic parts in real space
//   W    [Ns][N][N][N] complex T     periodic parts of V_x psi
//   H    [chain][N][N][N] complex T  pair density after the plane pass
//   vq   [nq][N][N][N] T             v(G + q) / Ntot per distinct q
//   vq64 [nq][N][N][N] double        v(G + q)
#pragma once

#include "fock_kernels.cuh"

namespace fockx {

// X[q] = scatter(c_{band0 + q}) on the sphere of one k point (X zeroed before).
template <class T>
__global__ void k_scatter_k(int npw, const int* __restrict__ gidx, int64_t ntot,
                            const double2* __restrict__ psiG, int band0, cplx<T>* __restrict__ X) {
  const int q = blockIdx.y;
  cplx<T>* Xq = X + (int64_t)q * ntot;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < npw; k += gridDim.x * blockDim.x) {
    const double2 c = psiG[(int64_t)(band0 + q) * npw + k];
    Xq[gidx[k]] = cmake<T>(T(c.x), T(c.y));
  }
}

// 2D FFT of plane i1 of X[q].  MODE 0: X -> u[band0 + q] * psi_scale (inverse
// transform of the orbitals); MODE 1: W[band0 + q] -> X (forward transform of V_x psi).
template <class T, int N, int SIGN, int MODE>
__global__ void __launch_bounds__(Geo<T, N>::THR_PLANE)
    k_plane_k(DevPlan g, cplx<T>* __restrict__ X, cplx<T>* __restrict__ U, int band0) {
  using C = cplx<T>;
  using G = Geo<T, N>;
  constexpr int RP = G::RP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* P = reinterpret_cast<C*>(smem_raw);
  C* tw = P + N * RP;
  const int i1 = blockIdx.x, q = blockIdx.y;
  const int64_t plane0 = (int64_t)i1 * N * N;
  C* Xq = X + (int64_t)q * g.ntot + plane0;
  C* Ub = U + (int64_t)(band0 + q) * g.ntot + plane0;
  load_twiddles<T>(tw, g);
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i2 = e / N, i3 = e - i2 * N;
    P[i2 * RP + i3] = MODE == 0 ? Xq[e] : Ub[e];
  }
  __syncthreads();
  fft_lines<T, N, SIGN, N, G::TLP, RP, 1>(P, tw);  // along i3
  fft_lines<T, N, SIGN, N, G::TLP, 1, RP>(P, tw);  // along i2
  const T s = T(g.psi_scale);
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i2 = e / N, i3 = e - i2 * N;
    const C z = P[i2 * RP + i3];
    if (MODE == 0) Ub[e] = cmake<T>(z.x * s, z.y * s);
    else Xq[e] = z;
  }
}

// (V_x psi)(G) of band band0 + q on the sphere of one k point.
template <class T>
__global__ void k_gather_k(int npw, const int* __restrict__ gidx, int64_t ntot, double scale,
                           const cplx<T>* __restrict__ X, int band0, double2* __restrict__ vpsiG) {
  const int q = blockIdx.y;
  const cplx<T>* Xq = X + (int64_t)q * ntot;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < npw; k += gridDim.x * blockDim.x) {
    const cplx<T> y = Xq[gidx[k]];
    vpsiG[(int64_t)(band0 + q) * npw + k] = make_double2(scale * double(y.x), scale * double(y.y));
  }
}

// Forward plane pass of a pair: plane i1 of u_a* u_b, 2D FFT, whole plane to H.
template <class T, int N>
__global__ void __launch_bounds__(Geo<T, N>::THR_PLANE)
    k_kpair_fwd(DevPlan g, const cplx<T>* __restrict__ u, const Chain* __restrict__ chains,
                cplx<T>* __restrict__ H) {
  using C = cplx<T>;
  using G = Geo<T, N>;
  constexpr int RP = G::RP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* P = reinterpret_cast<C*>(smem_raw);
  C* tw = P + N * RP;
  const int i1 = blockIdx.x;
  const Chain ch = chains[blockIdx.y];
  load_twiddles<T>(tw, g);
  const int64_t plane0 = (int64_t)i1 * N * N;
  const C* ua = u + (int64_t)ch.ai * g.ntot + plane0;
  const C* ub = u + (int64_t)ch.aj * g.ntot + plane0;
  // columns first, the first stage reading conj(u_a) u_b straight from global
  // memory (consecutive columns per warp: coalesced), then the rows
  const auto product = [&](int i3, int i2) {
    const int e = i2 * N + i3;
    const C a = ua[e], b = ub[e];
    return cmake<T>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);  // conj(a) b
  };
  fft_lines_from<T, N, -1, N, G::TLP, 1, RP, kMaxThreads>(P, tw, product);  // along i2
  fft_lines<T, N, -1, N, G::TLP, RP, 1>(P, tw);                            // along i3
  C* Hp = H + (int64_t)blockIdx.y * g.ntot + plane0;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i2 = e / N, i3 = e - i2 * N;
    Hp[e] = P[i2 * RP + i3];
  }
}

// Column pass of a pair: row k2, FFT along i1, times v(G + q) / Ntot, energy
// partial sum_G v(G + q) |rho(G)|^2, inverse FFT along k1.
template <class T, int N>
__global__ void __launch_bounds__(Geo<T, N>::THR_COLF, Geo<T, N>::MIN_CTAS)
    k_kpair_col(DevPlan g, cplx<T>* __restrict__ H, const Chain* __restrict__ chains,
                double* __restrict__ epair) {
  using C = cplx<T>;
  using G = Geo<T, N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* S = reinterpret_cast<C*>(smem_raw);
  C* tw = S + N * N;
  double* red = reinterpret_cast<double*>(tw + G::TWN);
  const int k2 = blockIdx.x;
  const Chain ch = chains[blockIdx.y];
  C* Hc = H + (int64_t)blockIdx.y * g.ntot;
  load_twiddles<T>(tw, g);
  // the row k2 of every plane i1, read by the first stage of the transform
  // along i1 straight from global memory
  const auto val = [&](int i3, int i1) { return Hc[((int64_t)i1 * N + k2) * N + i3]; };
  fft_lines_from<T, N, -1, N, G::TLP, 1, N, kMaxThreads>(S, tw, val);  // along i1
  const int64_t qoff = (int64_t)ch.pad1 * g.ntot;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if constexpr (sizeof(T) == 8) {
    const double* v64 = g.vtabq64 + qoff;
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
      const int k1 = e / N, k3 = e - k1 * N;
      const double v = v64[((int64_t)k1 * N + k2) * N + k3];
      C z = S[e];
      acc[0] += v * (z.x * z.x + z.y * z.y);
      const double vs = v * g.inv_ntot;
      z.x *= vs;
      z.y *= vs;
      S[e] = z;
    }
  } else {
    const T* vt = static_cast<const T*>(g.vtabq) + qoff;  // v / Ntot
    float accf[4] = {0.f, 0.f, 0.f, 0.f};
    // the terms with |m + q|^2 <= msmall2 (reduced coordinates) in FP64 from
    // the FP64 table; the one with m + q = 0 (q = 0 pairs) from the FP64
    // overlap of the pair's coefficients when the plan provides it
    bool row_small = false;
    float q1 = 0.f, q3 = 0.f, r2 = 0.f;
    if (g.qfrac != nullptr && g.msmall2 >= 0) {
      q1 = g.qfrac[3 * ch.pad1];
      q3 = g.qfrac[3 * ch.pad1 + 2];
      const float m2 = float(freq_of(k2, N)) + g.qfrac[3 * ch.pad1 + 1];
      r2 = m2 * m2;
      row_small = r2 <= float(g.msmall2);
    }
    if (!row_small) {
      for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int k1 = e / N, k3 = e - k1 * N;
        const T v = vt[((int64_t)k1 * N + k2) * N + k3];
        C z = S[e];
        accf[0] += v * (z.x * z.x + z.y * z.y);
        z.x *= v;
        z.y *= v;
        S[e] = z;
      }
    } else {
      const double* v64 = g.vtabq64 + qoff;
      double e64 = 0.0;
      // |m1 + q1|^2 <= msmall2 - m2q^2 bounds |m1| by b1 (and m3 by b3): an
      // integer box test first, the exact one inside it; k3 is the same for
      // all of a thread's elements when the CTA's threads are a multiple of N
      const float lim = sqrtf(float(g.msmall2) - r2);
      const int b1 = min(N / 2 - 1, (int)floorf(lim + fabsf(q1))), b3 = min(N / 2 - 1, (int)floorf(lim + fabsf(q3)));
      const bool k3_fixed = blockDim.x % N == 0;
      const int k3t = threadIdx.x % N;
      const bool box3_t = (k3t + b3 < N ? k3t + b3 : k3t + b3 - N) <= 2 * b3;
      for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int k1 = e / N, k3 = e - k1 * N;
        const int64_t vi = ((int64_t)k1 * N + k2) * N + k3;
        C z = S[e];
        const int w1 = k1 + b1 < N ? k1 + b1 : k1 + b1 - N;
        const bool box3 = k3_fixed ? box3_t : (k3 + b3 < N ? k3 + b3 : k3 + b3 - N) <= 2 * b3;
        bool small = false;
        if (box3 && w1 <= 2 * b1) {
          const float m1 = float(freq_of(k1, N)) + q1, m3 = float(freq_of(k3, N)) + q3;
          small = m1 * m1 + r2 + m3 * m3 <= float(g.msmall2);
        }
        if (small) {
          double zx = z.x, zy = z.y;
          if (g.kovl_re != nullptr && ch.pad1 == g.q0 && k1 == 0 && k2 == 0 && k3 == 0 &&
              ch.ai / g.kovl_nb == ch.aj / g.kovl_nb) {
            // q = 0 pair (a, b) of one k point: sum over the grid of conj(u_a) u_b
            const int nb = g.kovl_nb, kk = ch.ai / nb;
            const int64_t oi = ((int64_t)kk * nb + ch.ai % nb) * nb + ch.aj % nb;
            zx = g.ovl_scale * g.kovl_re[oi];
            zy = g.ovl_scale * g.kovl_im[oi];
          }
          const double v = v64[vi];
          e64 += v * (zx * zx + zy * zy);
          const double vs = v * g.inv_ntot;
          z.x = T(zx * vs);
          z.y = T(zy * vs);
        } else {
          const T v = vt[vi];
          accf[0] += v * (z.x * z.x + z.y * z.y);
          z.x *= v;
          z.y *= v;
        }
        S[e] = z;
      }
      if (e64 != 0.0 && ch.pa >= 0) atomicAdd(&epair[ch.pa], e64);
    }
    float hi[4], lo[4];
    block_sum4_ff(accf, hi, lo, reinterpret_cast<float*>(red));
    if (threadIdx.x == 0) acc[0] = ((double)hi[0] + (double)lo[0]) * double(g.ntot);
  }
  __syncthreads();
  fft_lines<T, N, +1, N, G::TLP, 1, N>(S, tw);  // inverse along k1
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i1 = e / N, i3 = e - i1 * N;
    Hc[((int64_t)i1 * N + k2) * N + i3] = S[e];
  }
  if constexpr (sizeof(T) == 8) block_sum4(acc, red);
  if (threadIdx.x == 0 && ch.pa >= 0) atomicAdd(&epair[ch.pa], acc[0]);
}

// Inverse plane pass of a pair and the W updates.
template <class T, int N>
__global__ void __launch_bounds__(Geo<T, N>::THR_PLANE, Geo<T, N>::MIN_CTAS_KINV)
    k_kpair_inv(DevPlan g, const cplx<T>* __restrict__ u, cplx<T>* __restrict__ W,
                const T* __restrict__ occw, const Chain* __restrict__ chains, const cplx<T>* __restrict__ H) {
  using C = cplx<T>;
  using G = Geo<T, N>;
  constexpr int RP = G::RP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* P = reinterpret_cast<C*>(smem_raw);
  C* tw = P + N * RP;
  const int i1 = blockIdx.x;
  const Chain ch = chains[blockIdx.y];
  load_twiddles<T>(tw, g);
  const int64_t plane0 = (int64_t)i1 * N * N;
  const C* Hp = H + (int64_t)blockIdx.y * g.ntot + plane0;
  // the plane, read by the first stage of the transform along k2 straight from
  // global memory (consecutive columns k3 per warp), then the rows
  const auto val = [&](int k3, int k2) { return Hp[k2 * N + k3]; };
  fft_lines_from<T, N, +1, N, G::TLP, 1, RP, kMaxThreads>(P, tw, val);  // along k2
  fft_lines<T, N, +1, N, G::TLP, RP, 1>(P, tw);                        // along k3
  const int a = ch.ai, b = ch.aj;
  const bool both = a != b;
  const T fa = occw[a], fb = occw[b];
  const C* ua = u + (int64_t)a * g.ntot + plane0;
  const C* ub = u + (int64_t)b * g.ntot + plane0;
  C* wa = W + (int64_t)a * g.ntot + plane0;
  C* wb = W + (int64_t)b * g.ntot + plane0;
  if constexpr (sizeof(T) == 4) {
    static_assert(N % 2 == 0, "pairwise vector updates need even N");
    // two complex points per thread: one 16-byte vector atomic per target
    for (int e2 = threadIdx.x; e2 < N * N / 2; e2 += blockDim.x) {
      const int e = 2 * e2;
      const int i2 = e / N, i3 = e - i2 * N;
      const C p0 = P[i2 * RP + i3], p1 = P[i2 * RP + i3 + 1];
      const float4 va = *reinterpret_cast<const float4*>(ua + e);
      float4 d;  // -fa * ua * phi
      d.x = -fa * (va.x * p0.x - va.y * p0.y);
      d.y = -fa * (va.x * p0.y + va.y * p0.x);
      d.z = -fa * (va.z * p1.x - va.w * p1.y);
      d.w = -fa * (va.z * p1.y + va.w * p1.x);
      asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(reinterpret_cast<float*>(wb + e)),
                   "f"(d.x), "f"(d.y), "f"(d.z), "f"(d.w)
                   : "memory");
      if (both) {
        const float4 vb = *reinterpret_cast<const float4*>(ub + e);
        float4 f;  // -fb * ub * conj(phi)
        f.x = -fb * (vb.x * p0.x + vb.y * p0.y);
        f.y = -fb * (vb.y * p0.x - vb.x * p0.y);
        f.z = -fb * (vb.z * p1.x + vb.w * p1.y);
        f.w = -fb * (vb.w * p1.x - vb.z * p1.y);
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(reinterpret_cast<float*>(wa + e)),
                     "f"(f.x), "f"(f.y), "f"(f.z), "f"(f.w)
                     : "memory");
      }
    }
  } else {
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
      const int i2 = e / N, i3 = e - i2 * N;
      const C p = P[i2 * RP + i3];
      const C x = ua[e];
      atomicAdd(&wb[e].x, -fa * (x.x * p.x - x.y * p.y));
      atomicAdd(&wb[e].y, -fa * (x.x * p.y + x.y * p.x));
      if (both) {
        const C y = ub[e];
        atomicAdd(&wa[e].x, -fb * (y.x * p.x + y.y * p.y));
        atomicAdd(&wa[e].y, -fb * (y.y * p.x - y.x * p.y));
      }
    }
  }
}

template <class T, int N>
struct LaunchK {
  using C = cplx<T>;
  using G = Geo<T, N>;

  static cudaError_t configure() {
    const void* fns[] = {(const void*)k_plane_k<T, N, +1, 0>, (const void*)k_plane_k<T, N, -1, 1>,
                         (const void*)k_kpair_fwd<T, N>, (const void*)k_kpair_inv<T, N>,
                         (const void*)k_col_full<T, N, +1>, (const void*)k_col_full<T, N, -1>};
    for (const void* f : fns) {
      cudaError_t err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)G::SMEM_PLANE);
      if (err != cudaSuccess) return err;
    }
    return cudaFuncSetAttribute((const void*)k_kpair_col<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_colk());
  }

  static constexpr size_t smem_colk() { return sizeof(C) * (size_t)(N * N + G::TWN) + 32 * 4 * sizeof(double); }

  static cudaError_t to_real(const DevPlan& g, const double2* psiG, int npw, const int* gidx, int band0,
                             int nbat, void* Xv, void* u, cudaStream_t s) {
    C* X = static_cast<C*>(Xv);
    cudaError_t err = cudaMemsetAsync(X, 0, sizeof(C) * (size_t)g.ntot * nbat, s);
    if (err != cudaSuccess) return err;
    k_scatter_k<T><<<dim3((npw + 255) / 256, nbat), 256, 0, s>>>(npw, gidx, g.ntot, psiG, 0, X);
    k_col_full<T, N, +1><<<dim3(N, nbat), G::THR_COLF, G::SMEM_COLF, s>>>(g, X);
    k_plane_k<T, N, +1, 0><<<dim3(N, nbat), G::THR_PLANE, G::SMEM_PLANE, s>>>(g, X, static_cast<C*>(u), band0);
    return cudaGetLastError();
  }

  static cudaError_t pair_fwd(const DevPlan& g, const void* u, const Chain* ch, int nch, void* H,
                              cudaStream_t s) {
    k_kpair_fwd<T, N><<<dim3(N, nch), G::THR_PLANE, G::SMEM_PLANE, s>>>(g, static_cast<const C*>(u), ch,
                                                                      static_cast<C*>(H));
    return cudaGetLastError();
  }

  static cudaError_t pair_col(const DevPlan& g, void* H, const Chain* ch, int nch, double* ep,
                              cudaStream_t s) {
    k_kpair_col<T, N><<<dim3(N, nch), G::THR_COLF, smem_colk(), s>>>(g, static_cast<C*>(H), ch, ep);
    return cudaGetLastError();
  }

  static cudaError_t pair_inv(const DevPlan& g, const void* u, void* W, const void* occw, const Chain* ch,
                              int nch, const void* H, cudaStream_t s) {
    k_kpair_inv<T, N><<<dim3(N, nch), G::THR_PLANE, G::SMEM_PLANE, s>>>(
        g, static_cast<const C*>(u), static_cast<C*>(W), static_cast<const T*>(occw), ch,
        static_cast<const C*>(H));
    return cudaGetLastError();
  }

  static cudaError_t to_sphere(const DevPlan& g, const void* W, int band0, int nbat, int npw, const int* gidx,
                               void* Xv, double2* vpsiG, cudaStream_t s) {
    C* X = static_cast<C*>(Xv);
    k_plane_k<T, N, -1, 1><<<dim3(N, nbat), G::THR_PLANE, G::SMEM_PLANE, s>>>(
        g, X, const_cast<C*>(static_cast<const C*>(W)), band0);
    k_col_full<T, N, -1><<<dim3(N, nbat), G::THR_COLF, G::SMEM_COLF, s>>>(g, X);
    k_gather_k<T><<<dim3((npw + 255) / 256, nbat), 256, 0, s>>>(npw, gidx, g.ntot, g.out_scale, X, 0, vpsiG);
    return cudaGetLastError();
  }

  static constexpr KOps ops() {
    return KOps{configure, to_real, pair_fwd, pair_col, pair_inv, to_sphere};
  }
};

}  // namespace fockx
