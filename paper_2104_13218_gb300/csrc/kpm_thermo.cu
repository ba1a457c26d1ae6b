// Thermodynamics from Chebyshev moments: Jackson kernel (Eq. E-2-8), the
// weights gamma_k of the Gauss-Chebyshev quadrature (Eq. quad and the
// expression of gamma_k that follows it), and the sector sum of the
// partition function with E, C (Eq. E-2-2-B) and chi (Eq. E-2-2-C).  All FP64.
//
// gamma_k is evaluated as a direct sum over n with cos(n pi (k+1/2)/Nq)
// read from a table of cos(pi j / (2 Nq)), j = n (2k+1) mod 4 Nq, which is
// exact in the index arithmetic (the paper's DCT-III gives the same values
// faster; here K * Nq is at most a few million per sector).  The Boltzmann
// factors are shifted by the lowest quadrature energy E_ref so that low
// temperatures do not underflow.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kpm_device.cuh"

namespace kpm {

constexpr double kPi = 3.14159265358979323846;

// The quadrature sums run over "entries": one per sector, or two for a
// sector that stands for +M and -M (mirror) in a magnetic field, where the
// two members' energies differ.  Entry e belongs to sector e_sec[e], has
// weight factor e_fac[e] = mult * dim / Nq, shift e_b[e] = b + h M (Zeeman
// term of Eq. E-3-1-1 with h = g mu_B B) and sign e_sm[e] of its
// magnetisation relative to the sector's moments mu_M (+1; -1 for the -M
// member; 0 for a mirrored pair at zero field, whose <M> terms cancel).
struct ThermoArgs {
  const double *mu[3];    // mu, mu_M, mu_M2 [S][K]
  const double *gk;       // g_n [K]
  const double *ctab;     // cos(pi j/(2 Nq)), j < 4 Nq
  double *gamma;          // [S][3][Nq]
  const double *a;        // [S]
  int nE;                 // entries
  const int *e_sec;       // [nE]
  const double *e_fac, *e_b, *e_sm;  // [nE]
  const int *s_estart;    // [S+1]: entries of sector s (entries are in sector order)
  const double *T;        // [nT]
  double *out[5];         // lnZ, signZ, E, C, chi [nT]
  double *stats;          // [nT][5]: S0, Ebar, C, <M>, <M^2>
  double *u;              // [S][3][Nq] backward
  const double *cot[4];   // dL/dlnZ, dL/dE, dL/dC, dL/dchi [nT] (may be NULL)
  double *grad[3];        // dL/dmu, dL/dmu_M, dL/dmu_M2 [S][K]
  int S, K, Nq, nT;
  double e_ref;
};

__global__ void thermo_tables_kernel(double *gk, double *ctab, int K, int Nq, int jackson) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < K) {
    double g = 1.0;
    if (jackson) {
      const double q = kPi / (K + 1);
      g = ((K - i + 1) * cos(q * i) + sin(q * i) / tan(q)) / (K + 1);
    }
    gk[i] = g;
  }
  if (i < 4 * Nq) ctab[i] = cos(kPi * i / (2.0 * Nq));
}

__device__ __forceinline__ double cos_nk(const double *ctab, int n, int k, int Nq) {
  const int64_t j = ((int64_t)n * (2 * k + 1)) % (4 * (int64_t)Nq);
  return ctab[j];
}

// gamma[s][q][k] = g_0 mu_0 + 2 sum_{n>=1} g_n mu_n cos(n theta_k)
__global__ void thermo_gamma_kernel(const __grid_constant__ ThermoArgs a) {
  const int total = a.S * 3 * a.Nq;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int s = i / (3 * a.Nq);
    const int q = (i / a.Nq) % 3;
    const int k = i % a.Nq;
    const double *m = a.mu[q] + (int64_t)s * a.K;
    double acc = a.gk[0] * m[0];
    for (int n = 1; n < a.K; ++n) acc = fma(2.0 * a.gk[n] * m[n], cos_nk(a.ctab, n, k, a.Nq), acc);
    a.gamma[i] = acc;
  }
}

template <int NQ>
__device__ __forceinline__ void block_sum_any(double (&v)[NQ], double *scratch) {
  block_sum<NQ>(v, scratch);
}

// One block per temperature: the shifted Boltzmann sums and the observables.
__global__ void __launch_bounds__(kThreads) thermo_sums_kernel(const __grid_constant__ ThermoArgs a) {
  __shared__ double s_red[kWarps * 4];
  __shared__ double s_b[4];
  const int it = blockIdx.x;
  const double beta = 1.0 / a.T[it];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const int total = a.nE * a.Nq;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int en = i / a.Nq, k = i % a.Nq;
    const int s = a.e_sec[en];
    const double x = cos(kPi * (k + 0.5) / a.Nq);
    const double E = a.a[s] * x + a.e_b[en];
    const double e = a.e_fac[en] * exp(-beta * (E - a.e_ref));
    const double *g = a.gamma + (int64_t)s * 3 * a.Nq;
    const double w = e * g[k];
    v[0] += w;
    v[1] += w * E;
    v[2] += a.e_sm[en] * e * g[a.Nq + k];
    v[3] += e * g[2 * a.Nq + k];
  }
  block_sum<4>(v, s_red);
  if (threadIdx.x == 0) {
    for (int q = 0; q < 4; ++q) s_b[q] = v[q];
  }
  __syncthreads();
  const double S0 = s_b[0];
  const double Ebar = s_b[1] / S0;
  double c[1] = {0.0};
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int en = i / a.Nq, k = i % a.Nq;
    const int s = a.e_sec[en];
    const double x = cos(kPi * (k + 0.5) / a.Nq);
    const double E = a.a[s] * x + a.e_b[en];
    const double e = a.e_fac[en] * exp(-beta * (E - a.e_ref));
    const double w = e * a.gamma[(int64_t)s * 3 * a.Nq + k];
    const double dE = E - Ebar;
    c[0] += w * dE * dE;
  }
  block_sum<1>(c, s_red);
  if (threadIdx.x == 0) {
    const double M1 = s_b[2] / S0, M2 = s_b[3] / S0;
    const double C = beta * beta * c[0] / S0;
    const double chi = beta * (M2 - M1 * M1);
    if (a.out[0]) a.out[0][it] = log(fabs(S0)) - beta * a.e_ref;
    if (a.out[1]) a.out[1][it] = S0 > 0 ? 1.0 : (S0 < 0 ? -1.0 : 0.0);
    if (a.out[2]) a.out[2][it] = Ebar;
    if (a.out[3]) a.out[3][it] = C;
    if (a.out[4]) a.out[4][it] = chi;
    if (a.stats) {
      double *st = a.stats + (int64_t)it * 5;
      st[0] = S0;
      st[1] = Ebar;
      st[2] = C;
      st[3] = M1;
      st[4] = M2;
    }
  }
}

// u[s][q][k] = sum_T (dL/dw^(q)_k(T)) * fac_s exp(-beta_T (E_k - E_ref))
__global__ void thermo_u_kernel(const __grid_constant__ ThermoArgs a) {
  const int total = a.S * a.Nq;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int s = i / a.Nq, k = i % a.Nq;
    const double x = cos(kPi * (k + 0.5) / a.Nq);
    double u0 = 0.0, u1 = 0.0, u2 = 0.0;
    for (int en = a.s_estart[s]; en < a.s_estart[s + 1]; ++en) {
    const double E = a.a[s] * x + a.e_b[en];
    for (int it = 0; it < a.nT; ++it) {
      const double beta = 1.0 / a.T[it];
      const double *st = a.stats + (int64_t)it * 5;
      const double S0 = st[0], Eb = st[1], C = st[2], M1 = st[3], M2 = st[4];
      const double lz = a.cot[0] ? a.cot[0][it] : 0.0;
      const double le = a.cot[1] ? a.cot[1][it] : 0.0;
      const double lc = a.cot[2] ? a.cot[2][it] : 0.0;
      const double lx = a.cot[3] ? a.cot[3][it] : 0.0;
      const double e = a.e_fac[en] * exp(-beta * (E - a.e_ref));
      const double dE = E - Eb;
      const double A = (lz + le * dE + lc * (beta * beta * dE * dE - C) +
                        lx * beta * (2.0 * M1 * M1 - M2)) / S0;
      const double B = -2.0 * lx * beta * M1 / S0;
      const double Cc = lx * beta / S0;
      u0 += A * e;
      u1 += a.e_sm[en] * B * e;
      u2 += Cc * e;
    }
    }
    double *u = a.u + (int64_t)s * 3 * a.Nq;
    u[k] = u0;
    u[a.Nq + k] = u1;
    u[2 * a.Nq + k] = u2;
  }
}

// dL/dmu^(q)_n = g_n c_n sum_k cos(n theta_k) u^(q)_k, c_0 = 1, c_n = 2
__global__ void thermo_grad_kernel(const __grid_constant__ ThermoArgs a) {
  const int total = a.S * 3 * a.K;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int s = i / (3 * a.K);
    const int q = (i / a.K) % 3;
    const int n = i % a.K;
    if (!a.grad[q]) continue;
    const double *u = a.u + ((int64_t)s * 3 + q) * a.Nq;
    double acc = 0.0;
    for (int k = 0; k < a.Nq; ++k) acc = fma(cos_nk(a.ctab, n, k, a.Nq), u[k], acc);
    a.grad[q][(int64_t)s * a.K + n] = a.gk[n] * (n == 0 ? 1.0 : 2.0) * acc;
  }
}

namespace {

struct ThermoCall {
  ThermoArgs a;
  std::vector<double> host;  // entry tables staged for the copies (kept until the call ends)
  std::vector<int> ihost;
  void *scratch = nullptr;
  cudaStream_t stream = nullptr;
  ~ThermoCall() {
    if (scratch) {
      cudaFreeAsync(scratch, stream);
      cudaStreamSynchronize(stream);
    }
  }
};

int setup_thermo(ThermoCall &tc, int S, int K, const double *mu, const double *mu_M,
                 const double *mu_M2, const double *dim, const int32_t *mirror, const double *Mv,
                 const double *a, const double *b, double field, int kernel, int n_quad, int nT,
                 const double *T, int on_device, bool backward, cudaStream_t stream) {
  KPM_REQUIRE(S >= 1 && K >= 1 && nT >= 1, KPM_EINVAL, "need S, K, n_T >= 1");
  KPM_REQUIRE(mu && dim && a && b && T, KPM_EINVAL, "NULL input");
  KPM_REQUIRE(kernel == KPM_KERNEL_NONE || kernel == KPM_KERNEL_JACKSON, KPM_EINVAL, "kernel %d",
              kernel);
  const int Nq = n_quad > 0 ? n_quad : K;
  KPM_REQUIRE(Nq <= (1 << 20), KPM_EINVAL, "n_quad too large");
  for (int i = 0; i < S; ++i)
    KPM_REQUIRE(a[i] > 0 && std::isfinite(a[i]) && std::isfinite(b[i]) && dim[i] > 0, KPM_EINVAL,
                "sector %d: a = %g, b = %g, dim = %g", i, a[i], b[i], dim[i]);
  for (int i = 0; i < nT; ++i) KPM_REQUIRE(T[i] > 0, KPM_EINVAL, "T[%d] = %g <= 0", i, T[i]);
  KPM_REQUIRE(std::isfinite(field), KPM_EINVAL, "field = %g", field);
  KPM_REQUIRE(field == 0.0 || Mv != nullptr, KPM_EINVAL,
              "a magnetic field needs the magnetisation M of every sector");
  if (field != 0.0)
    for (int i = 0; i < S; ++i)
      KPM_REQUIRE(std::isfinite(Mv[i]), KPM_EINVAL,
                  "sector %d: a magnetic field needs S^z sectors (M varies inside a full-space run)",
                  i);
  // quadrature entries: one per sector, two for a mirrored pair in a field
  std::vector<int> e_sec, s_estart(S + 1);
  std::vector<double> e_fac, e_b, e_sm;
  for (int i = 0; i < S; ++i) {
    s_estart[i] = (int)e_sec.size();
    const bool mir = mirror && mirror[i];
    const double M = (Mv && std::isfinite(Mv[i])) ? Mv[i] : 0.0;
    if (mir && field != 0.0) {
      for (int sgn : {1, -1}) {
        e_sec.push_back(i);
        e_fac.push_back(dim[i] / Nq);
        e_b.push_back(b[i] + field * sgn * M);
        e_sm.push_back((double)sgn);
      }
    } else {
      e_sec.push_back(i);
      e_fac.push_back((mir ? 2.0 : 1.0) * dim[i] / Nq);
      e_b.push_back(b[i] + field * M);
      e_sm.push_back(mir ? 0.0 : 1.0);
    }
  }
  s_estart[S] = (int)e_sec.size();
  const int nE = (int)e_sec.size();
  tc.stream = stream;
  const size_t SK = (size_t)S * K;
  const size_t bytes = align256(K * 8) + align256(4 * (size_t)Nq * 8) + align256(S * 3 * (size_t)Nq * 8) +
                       align256(S * 8) + 3 * align256(nE * 8) + align256(nE * 4) +
                       align256((S + 1) * 4) + align256(nT * 8) +
                       align256(nT * 5 * 8) + (backward ? align256(S * 3 * (size_t)Nq * 8) : 0) +
                       5 * align256(SK * 8) + 4096;
  KPM_CUDA(cudaMallocAsync(&tc.scratch, bytes, stream));
  Arena ar{reinterpret_cast<char *>(tc.scratch), bytes, 0};
  ThermoArgs &A = tc.a;
  A = ThermoArgs{};
  A.S = S;
  A.K = K;
  A.Nq = Nq;
  A.nT = nT;
  double *gk = ar.take<double>(K);
  double *ctab = ar.take<double>(4 * (size_t)Nq);
  A.gk = gk;
  A.ctab = ctab;
  A.gamma = ar.take<double>((size_t)S * 3 * Nq);
  double *da = ar.take<double>(S);
  double *dfac = ar.take<double>(nE);
  double *deb = ar.take<double>(nE);
  double *desm = ar.take<double>(nE);
  int *desec = ar.take<int>(nE);
  int *dstart = ar.take<int>(S + 1);
  double *dT = ar.take<double>(nT);
  A.stats = ar.take<double>((size_t)nT * 5);
  if (backward) A.u = ar.take<double>((size_t)S * 3 * Nq);
  double e_ref = INFINITY;
  const double xmax = std::cos(kPi * 0.5 / Nq);
  for (int en = 0; en < nE; ++en) e_ref = std::min(e_ref, e_b[en] - a[e_sec[en]] * xmax);
  A.e_ref = e_ref;
  tc.host.assign(e_fac.begin(), e_fac.end());
  tc.host.insert(tc.host.end(), e_b.begin(), e_b.end());
  tc.host.insert(tc.host.end(), e_sm.begin(), e_sm.end());
  tc.ihost.assign(e_sec.begin(), e_sec.end());
  tc.ihost.insert(tc.ihost.end(), s_estart.begin(), s_estart.end());
  KPM_CUDA(cudaMemcpyAsync(da, a, S * 8, cudaMemcpyHostToDevice, stream));
  KPM_CUDA(cudaMemcpyAsync(dfac, tc.host.data(), nE * 8, cudaMemcpyHostToDevice, stream));
  KPM_CUDA(cudaMemcpyAsync(deb, tc.host.data() + nE, nE * 8, cudaMemcpyHostToDevice, stream));
  KPM_CUDA(cudaMemcpyAsync(desm, tc.host.data() + 2 * nE, nE * 8, cudaMemcpyHostToDevice, stream));
  KPM_CUDA(cudaMemcpyAsync(desec, tc.ihost.data(), nE * 4, cudaMemcpyHostToDevice, stream));
  KPM_CUDA(cudaMemcpyAsync(dstart, tc.ihost.data() + nE, (S + 1) * 4, cudaMemcpyHostToDevice, stream));
  KPM_CUDA(cudaMemcpyAsync(dT, T, nT * 8, cudaMemcpyHostToDevice, stream));
  A.a = da;
  A.nE = nE;
  A.e_fac = dfac;
  A.e_b = deb;
  A.e_sm = desm;
  A.e_sec = desec;
  A.s_estart = dstart;
  A.T = dT;
  const double *ins[3] = {mu, mu_M, mu_M2};
  for (int q = 0; q < 3; ++q) {
    if (on_device || ins[q] == nullptr) {
      A.mu[q] = ins[q];
    } else {
      double *d = ar.take<double>(SK);
      KPM_CUDA(cudaMemcpyAsync(d, ins[q], SK * 8, cudaMemcpyHostToDevice, stream));
      A.mu[q] = d;
    }
  }
  // missing weighted moments: zeros
  for (int q = 1; q < 3; ++q) {
    if (A.mu[q] == nullptr) {
      double *d = ar.take<double>(SK);
      KPM_CUDA(cudaMemsetAsync(d, 0, SK * 8, stream));
      A.mu[q] = d;
    }
  }
  const int n = std::max(K, 4 * Nq);
  thermo_tables_kernel<<<(n + 255) / 256, 256, 0, stream>>>(gk, ctab, K, Nq,
                                                            kernel == KPM_KERNEL_JACKSON);
  KPM_CUDA(cudaGetLastError());
  const int total = S * 3 * Nq;
  thermo_gamma_kernel<<<std::min(4096, (total + 255) / 256), 256, 0, stream>>>(A);
  KPM_CUDA(cudaGetLastError());
  count_launches(2);
  return KPM_OK;
}

}  // namespace

}  // namespace kpm

using namespace kpm;

namespace kpm {
namespace {

int thermo_impl(int32_t n_sectors, int32_t n_moments, const double *mu, const double *mu_M,
                const double *mu_M2, const double *dim, const int32_t *mirror, const double *M,
                const double *a, const double *b, double field, int32_t kernel, int32_t n_quad,
                int32_t n_T, const double *T, double *lnZ, double *signZ, double *E, double *C,
                double *chi, int32_t on_device, cudaStream_t stream) {
  ThermoCall tc;
  KPM_TRY(setup_thermo(tc, n_sectors, n_moments, mu, mu_M, mu_M2, dim, mirror, M, a, b, field,
                       kernel, n_quad, n_T, T, on_device, false, stream));
  double *outs[5] = {lnZ, signZ, E, C, chi};
  std::vector<double> host(5 * (size_t)n_T);
  double *dev_out = nullptr;
  if (!on_device) {
    KPM_CUDA(cudaMallocAsync(&dev_out, 5 * (size_t)n_T * 8, stream));
    for (int q = 0; q < 5; ++q) tc.a.out[q] = dev_out + (size_t)q * n_T;
  } else {
    for (int q = 0; q < 5; ++q) tc.a.out[q] = outs[q];
  }
  thermo_sums_kernel<<<n_T, kThreads, 0, stream>>>(tc.a);
  KPM_CUDA(cudaGetLastError());
  count_launches(1);
  if (!on_device) {
    KPM_CUDA(cudaMemcpyAsync(host.data(), dev_out, 5 * (size_t)n_T * 8, cudaMemcpyDeviceToHost, stream));
    KPM_CUDA(cudaFreeAsync(dev_out, stream));
  }
  KPM_CUDA(cudaStreamSynchronize(stream));
  if (!on_device)
    for (int q = 0; q < 5; ++q)
      if (outs[q])
        for (int i = 0; i < n_T; ++i) outs[q][i] = host[(size_t)q * n_T + i];
  return KPM_OK;
}

int thermo_backward_impl(int32_t n_sectors, int32_t n_moments, const double *mu,
                         const double *mu_M, const double *mu_M2, const double *dim,
                         const int32_t *mirror, const double *M, const double *a, const double *b,
                         double field, int32_t kernel, int32_t n_quad, int32_t n_T,
                         const double *T, const double *dL_dlnZ, const double *dL_dE,
                         const double *dL_dC, const double *dL_dchi, double *dL_dmu,
                         double *dL_dmu_M, double *dL_dmu_M2, int32_t on_device,
                         cudaStream_t stream) {
  KPM_REQUIRE(dL_dmu != nullptr, KPM_EINVAL, "dL_dmu is NULL");
  ThermoCall tc;
  KPM_TRY(setup_thermo(tc, n_sectors, n_moments, mu, mu_M, mu_M2, dim, mirror, M, a, b, field,
                       kernel, n_quad, n_T, T, on_device, true, stream));
  const size_t SK = (size_t)n_sectors * n_moments;
  double *extra = nullptr;
  const double *cot_in[4] = {dL_dlnZ, dL_dE, dL_dC, dL_dchi};
  double *grads[3] = {dL_dmu, dL_dmu_M, dL_dmu_M2};
  KPM_CUDA(cudaMallocAsync(&extra, (4 * (size_t)n_T + 3 * SK) * 8 + 64, stream));
  for (int q = 0; q < 4; ++q) {
    if (!cot_in[q]) {
      tc.a.cot[q] = nullptr;
    } else if (on_device) {
      tc.a.cot[q] = cot_in[q];
    } else {
      double *d = extra + (size_t)q * n_T;
      KPM_CUDA(cudaMemcpyAsync(d, cot_in[q], n_T * 8, cudaMemcpyHostToDevice, stream));
      tc.a.cot[q] = d;
    }
  }
  for (int q = 0; q < 3; ++q) {
    if (!grads[q])
      tc.a.grad[q] = nullptr;
    else
      tc.a.grad[q] = on_device ? grads[q] : extra + 4 * (size_t)n_T + q * SK;
  }
  for (int q = 0; q < 5; ++q) tc.a.out[q] = nullptr;
  thermo_sums_kernel<<<n_T, kThreads, 0, stream>>>(tc.a);
  KPM_CUDA(cudaGetLastError());
  const int nu = n_sectors * tc.a.Nq;
  thermo_u_kernel<<<std::min(4096, (nu + 255) / 256), 256, 0, stream>>>(tc.a);
  KPM_CUDA(cudaGetLastError());
  const int ng = n_sectors * 3 * n_moments;
  thermo_grad_kernel<<<std::min(4096, (ng + 255) / 256), 256, 0, stream>>>(tc.a);
  KPM_CUDA(cudaGetLastError());
  count_launches(3);
  if (!on_device)
    for (int q = 0; q < 3; ++q)
      if (grads[q])
        KPM_CUDA(cudaMemcpyAsync(grads[q], tc.a.grad[q], SK * 8, cudaMemcpyDeviceToHost, stream));
  KPM_CUDA(cudaFreeAsync(extra, stream));
  KPM_CUDA(cudaStreamSynchronize(stream));
  return KPM_OK;
}

}  // namespace

// ---------------------------------------------------------------- realisations
// P realisations of the trace estimator from per-vector moments (Sec. 3,
// Eq. E-3-1 .. E-3-3): realisation p averages the moments of vectors
// p*R_per .. p*R_per + R_per - 1; its thermodynamics O_p(T) come from the
// same quadrature as kpm_thermo; then per temperature the mean
// O-bar = (1/P) sum_p O_p, the variance dO^2 = mean(O^2) - O-bar^2 and, with
// an exact curve, the systematic deviation |O-bar - O_E|.

// mu_p[p][s][n] = (1/R_per) sum_{r in p} mu_r[s][r][n]; mu_M = M mu, mu_M2 = M^2 mu.
__global__ void realisation_moments_kernel(const double *mu_r, const double *Ms, int S, int R,
                                           int R_per, int K, int P, double *mu_p, double *muM_p,
                                           double *muM2_p) {
  const int64_t total = (int64_t)P * S * K;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(i % K);
    const int s = (int)((i / K) % S);
    const int p = (int)(i / ((int64_t)K * S));
    double v = 0.0;
    for (int j = 0; j < R_per; ++j) v += mu_r[((int64_t)s * R + p * R_per + j) * K + n];
    v /= R_per;
    mu_p[i] = v;
    muM_p[i] = Ms[s] * v;
    muM2_p[i] = Ms[s] * Ms[s] * v;
  }
}

// all[p][q][t] (q: lnZ, E, C, chi) -> mean, var (Eq. E-3-1, E-3-2), dev (Eq. E-3-3).
__global__ void realisation_stats_kernel(const double *all, int P, int nT, const double *exact,
                                         double *mean, double *var, double *dev) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * nT) return;
  double s1 = 0.0, s2 = 0.0;
  for (int p = 0; p < P; ++p) {
    const double o = all[(int64_t)p * 4 * nT + i];
    s1 += o;
    s2 += o * o;
  }
  const double m = s1 / P;
  mean[i] = m;
  var[i] = s2 / P - m * m;
  if (dev != nullptr && exact != nullptr) dev[i] = fabs(m - exact[i]);
}

}  // namespace kpm

using namespace kpm;

extern "C" int kpm_thermo(int32_t n_sectors, int32_t n_moments, const double *mu,
                          const double *mu_M, const double *mu_M2, const double *dim,
                          const int32_t *mirror, const double *a, const double *b, int32_t kernel,
                          int32_t n_quad, int32_t n_T, const double *T, double *lnZ,
                          double *signZ, double *E, double *C, double *chi, int32_t on_device,
                          void *stream_ptr) {
  clear_error();
  return thermo_impl(n_sectors, n_moments, mu, mu_M, mu_M2, dim, mirror, nullptr, a, b, 0.0,
                     kernel, n_quad, n_T, T, lnZ, signZ, E, C, chi, on_device,
                     reinterpret_cast<cudaStream_t>(stream_ptr));
}

extern "C" int kpm_thermo_ex(int32_t n_sectors, int32_t n_moments, const double *mu,
                             const double *mu_M, const double *mu_M2, const double *dim,
                             const int32_t *mirror, const double *M, const double *a,
                             const double *b, double field, int32_t kernel, int32_t n_quad,
                             int32_t n_T, const double *T, double *lnZ, double *signZ, double *E,
                             double *C, double *chi, int32_t on_device, void *stream_ptr) {
  clear_error();
  return thermo_impl(n_sectors, n_moments, mu, mu_M, mu_M2, dim, mirror, M, a, b, field, kernel,
                     n_quad, n_T, T, lnZ, signZ, E, C, chi, on_device,
                     reinterpret_cast<cudaStream_t>(stream_ptr));
}

extern "C" int kpm_thermo_backward(int32_t n_sectors, int32_t n_moments, const double *mu,
                                   const double *mu_M, const double *mu_M2, const double *dim,
                                   const int32_t *mirror, const double *a, const double *b,
                                   int32_t kernel, int32_t n_quad, int32_t n_T, const double *T,
                                   const double *dL_dlnZ, const double *dL_dE,
                                   const double *dL_dC, const double *dL_dchi, double *dL_dmu,
                                   double *dL_dmu_M, double *dL_dmu_M2, int32_t on_device,
                                   void *stream_ptr) {
  clear_error();
  return thermo_backward_impl(n_sectors, n_moments, mu, mu_M, mu_M2, dim, mirror, nullptr, a, b,
                              0.0, kernel, n_quad, n_T, T, dL_dlnZ, dL_dE, dL_dC, dL_dchi, dL_dmu,
                              dL_dmu_M, dL_dmu_M2, on_device,
                              reinterpret_cast<cudaStream_t>(stream_ptr));
}

extern "C" int kpm_thermo_backward_ex(int32_t n_sectors, int32_t n_moments, const double *mu,
                                      const double *mu_M, const double *mu_M2, const double *dim,
                                      const int32_t *mirror, const double *M, const double *a,
                                      const double *b, double field, int32_t kernel,
                                      int32_t n_quad, int32_t n_T, const double *T,
                                      const double *dL_dlnZ, const double *dL_dE,
                                      const double *dL_dC, const double *dL_dchi,
                                      double *dL_dmu, double *dL_dmu_M, double *dL_dmu_M2,
                                      int32_t on_device, void *stream_ptr) {
  clear_error();
  return thermo_backward_impl(n_sectors, n_moments, mu, mu_M, mu_M2, dim, mirror, M, a, b, field,
                              kernel, n_quad, n_T, T, dL_dlnZ, dL_dE, dL_dC, dL_dchi, dL_dmu,
                              dL_dmu_M, dL_dmu_M2, on_device,
                              reinterpret_cast<cudaStream_t>(stream_ptr));
}

extern "C" int kpm_realisations(int32_t n_sectors, int32_t n_moments, int32_t R, int32_t R_per,
                                const double *mu_r, const double *dim, const int32_t *mirror,
                                const double *M, const double *a, const double *b, double field,
                                int32_t kernel, int32_t n_quad, int32_t n_T, const double *T,
                                const double *exact, double *mean, double *var, double *dev,
                                double *all, int32_t on_device, void *stream_ptr) {
  clear_error();
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_ptr);
  KPM_REQUIRE(mu_r && M && mean && var, KPM_EINVAL, "NULL argument");
  KPM_REQUIRE(n_sectors >= 1 && n_moments >= 1 && n_T >= 1, KPM_EINVAL, "empty problem");
  KPM_REQUIRE(R_per >= 1 && R >= R_per && R % R_per == 0, KPM_EINVAL,
              "R = %d is not a multiple of R_per = %d", R, R_per);
  for (int i = 0; i < n_sectors; ++i)
    KPM_REQUIRE(std::isfinite(M[i]), KPM_EINVAL,
                "sector %d: realisations need S^z sectors (finite M)", i);
  const int P = R / R_per;
  const size_t SK = (size_t)n_sectors * n_moments;
  const size_t PSK = (size_t)P * SK;
  const size_t P4T = (size_t)P * 4 * n_T;
  double *buf = nullptr;
  const size_t nbuf = (on_device ? 0 : (size_t)R * SK) + 3 * PSK + n_sectors + P4T + 5 * 4 * (size_t)n_T;
  KPM_CUDA(cudaMallocAsync(&buf, nbuf * 8, stream));
  struct Release {
    double *p;
    cudaStream_t s;
    ~Release() {
      cudaFreeAsync(p, s);
      cudaStreamSynchronize(s);
    }
  } release{buf, stream};
  double *d_mur = on_device ? const_cast<double *>(mu_r) : buf;
  double *mu_p = buf + (on_device ? 0 : (size_t)R * SK);
  double *muM_p = mu_p + PSK;
  double *muM2_p = muM_p + PSK;
  double *d_M = muM2_p + PSK;
  double *d_all = d_M + n_sectors;
  double *d_stats = d_all + P4T;  // mean, var, dev, exact, signZ scratch: [5][4][n_T]
  if (!on_device)
    KPM_CUDA(cudaMemcpyAsync(d_mur, mu_r, (size_t)R * SK * 8, cudaMemcpyHostToDevice, stream));
  KPM_CUDA(cudaMemcpyAsync(d_M, M, n_sectors * 8, cudaMemcpyHostToDevice, stream));
  {
    const int64_t tot = (int64_t)PSK;
    realisation_moments_kernel<<<(int)std::min<int64_t>(4096, (tot + 255) / 256), 256, 0, stream>>>(
        d_mur, d_M, n_sectors, R, R_per, n_moments, P, mu_p, muM_p, muM2_p);
    KPM_CUDA(cudaGetLastError());
    count_launches(1);
  }
  double *signz = d_stats + 4 * 4 * (size_t)n_T;
  for (int p = 0; p < P; ++p) {
    double *o = d_all + (size_t)p * 4 * n_T;  // lnZ, E, C, chi
    KPM_TRY(thermo_impl(n_sectors, n_moments, mu_p + p * SK, muM_p + p * SK, muM2_p + p * SK, dim,
                        mirror, M, a, b, field, kernel, n_quad, n_T, T, o, signz, o + n_T,
                        o + 2 * (size_t)n_T, o + 3 * (size_t)n_T, 1, stream));
  }
  double *d_mean = on_device ? mean : d_stats;
  double *d_var = on_device ? var : d_stats + 4 * (size_t)n_T;
  double *d_dev = dev ? (on_device ? dev : d_stats + 8 * (size_t)n_T) : nullptr;
  const double *d_exact = nullptr;
  if (exact) {
    if (on_device) {
      d_exact = exact;
    } else {
      double *e = d_stats + 12 * (size_t)n_T;
      KPM_CUDA(cudaMemcpyAsync(e, exact, 4 * (size_t)n_T * 8, cudaMemcpyHostToDevice, stream));
      d_exact = e;
    }
  }
  KPM_REQUIRE(dev == nullptr || exact != nullptr, KPM_EINVAL, "dev needs the exact curves");
  realisation_stats_kernel<<<(4 * n_T + 255) / 256, 256, 0, stream>>>(d_all, P, n_T, d_exact,
                                                                      d_mean, d_var, d_dev);
  KPM_CUDA(cudaGetLastError());
  count_launches(1);
  if (!on_device) {
    KPM_CUDA(cudaMemcpyAsync(mean, d_mean, 4 * (size_t)n_T * 8, cudaMemcpyDeviceToHost, stream));
    KPM_CUDA(cudaMemcpyAsync(var, d_var, 4 * (size_t)n_T * 8, cudaMemcpyDeviceToHost, stream));
    if (dev) KPM_CUDA(cudaMemcpyAsync(dev, d_dev, 4 * (size_t)n_T * 8, cudaMemcpyDeviceToHost, stream));
    if (all) KPM_CUDA(cudaMemcpyAsync(all, d_all, P4T * 8, cudaMemcpyDeviceToHost, stream));
  } else if (all) {
    KPM_CUDA(cudaMemcpyAsync(all, d_all, P4T * 8, cudaMemcpyDeviceToDevice, stream));
  }
  KPM_CUDA(cudaStreamSynchronize(stream));
  return KPM_OK;
}
