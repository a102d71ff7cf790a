// Geometry precompute of flexi_mesh_init, in FP64 (Sec. 3.1):
//  - tensor-product interpolation / differentiation along one direction
//    (generic 1-D operator applied to [B][nk][nj][ni] arrays),
//  - curl-form metric terms Ja^i_n = -xhat_i . curl_xi(x_l grad_xi x_m)
//    (Eq. contravariantBasisVectorsCurl) from the products v_j = x_l dx_m/dxi_j,
//  - Jacobian determinant, 1/J and the quadrature weights w_i w_j w_k J,
//  - face normals n = ntilde/|ntilde|, s_hat = |ntilde|, ntilde_d = +-Ja^l_d on the face.
#include "launch.h"

namespace flexi {

__global__ void k_apply1d(const double* __restrict__ in, double* __restrict__ out, const double* __restrict__ M,
                          int B, int ni, int nj, int nk, int l, int nout) {
  const int oi = l == 0 ? nout : ni, oj = l == 1 ? nout : nj, ok = l == 2 ? nout : nk;
  const long long tot = (long long)B * oi * oj * ok;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= tot) return;
  long long r = idx;
  const int i = r % oi; r /= oi;
  const int j = r % oj; r /= oj;
  const int k = r % ok; r /= ok;
  const long long b = r;
  const double* src = in + b * (long long)ni * nj * nk;
  const int nin = l == 0 ? ni : (l == 1 ? nj : nk);
  const int o = l == 0 ? i : (l == 1 ? j : k);
  double s = 0.0;
  for (int a = 0; a < nin; ++a) {
    const int ii = l == 0 ? a : i, jj = l == 1 ? a : j, kk = l == 2 ? a : k;
    s += M[o * nin + a] * src[(kk * nj + jj) * ni + ii];
  }
  out[idx] = s;
}

cudaError_t geom_apply1d(const double* in, double* out, const double* M, int B, int ni, int nj, int nk, int l,
                         int nout, cudaStream_t st) {
  const long long tot = (long long)B * (l == 0 ? nout : ni) * (l == 1 ? nout : nj) * (l == 2 ? nout : nk);
  k_apply1d<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(in, out, M, B, ni, nj, nk, l, nout);
  return cudaGetLastError();
}

// v[nn][j][e][node] = X[e][ll][node] * dX_j[e][m][node], (nn, m, ll) cyclic, dX_j = d x / d xi_j
__global__ void k_metric_products(const double* __restrict__ X, const double* __restrict__ dX0,
                                  const double* __restrict__ dX1, const double* __restrict__ dX2,
                                  double* __restrict__ v, int K, int n3) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = (long long)K * n3;
  if (idx >= tot) return;
  const long long e = idx / n3;
  const int node = idx % n3;
  const double* dX[3] = {dX0, dX1, dX2};
  for (int nn = 0; nn < 3; ++nn) {
    const int m = (nn + 1) % 3, ll = (nn + 2) % 3;
    const double xl = X[(e * 3 + ll) * n3 + node];
    for (int j = 0; j < 3; ++j) v[(nn * 3 + j) * tot + idx] = xl * dX[j][(e * 3 + m) * n3 + node];
  }
}

cudaError_t geom_metric_products(const double* XL, const double* const dXL[3], double* v, int K, int n3,
                                 cudaStream_t st) {
  const long long tot = (long long)K * n3;
  k_metric_products<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(XL, dXL[0], dXL[1], dXL[2], v, K, n3);
  return cudaGetLastError();
}

// Ja[e][i*3+nn] = -(dA - dB) where dA = D_{i+1} v_{i+2}, dB = D_{i+2} v_{i+1}
__global__ void k_curl(const double* __restrict__ dA, const double* __restrict__ dB, double* __restrict__ Ja, int K,
                       int n3, int i, int nn) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)K * n3) return;
  const long long e = idx / n3;
  const int node = idx % n3;
  Ja[(e * 9 + i * 3 + nn) * n3 + node] = -(dA[idx] - dB[idx]);
}

cudaError_t geom_curl(const double* dA, const double* dB, double* Ja, int K, int n3, int i, int nn, cudaStream_t st) {
  const long long tot = (long long)K * n3;
  k_curl<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(dA, dB, Ja, K, n3, i, nn);
  return cudaGetLastError();
}

// dX_l[e][c][node] = d x_c / d xi_l ; J = det; sJ = 1/J; wJ = w_i w_j w_k J
__global__ void k_jacobian(const double* __restrict__ dX0, const double* __restrict__ dX1,
                           const double* __restrict__ dX2, double* __restrict__ sJ, double* __restrict__ wJ,
                           const double* __restrict__ w, int K, int n, unsigned* __restrict__ bad) {
  const int n3 = n * n * n;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)K * n3) return;
  const long long e = idx / n3;
  const int node = idx % n3;
  const double* dX[3] = {dX0, dX1, dX2};
  double a[3][3];
  for (int c = 0; c < 3; ++c)
    for (int l = 0; l < 3; ++l) a[c][l] = dX[l][(e * 3 + c) * n3 + node];
  const double J = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                   a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
  if (!(J > 0.0)) atomicOr(bad, 1u);
  sJ[idx] = 1.0 / J;
  const int i = node % n, j = (node / n) % n, k = node / (n * n);
  wJ[idx] = w[i] * w[j] * w[k] * J;
}

cudaError_t geom_jacobian(const double* const dX[3], double* sJ, double* wJ, const double* w, int K, int n,
                          unsigned* bad, cudaStream_t st) {
  const long long tot = (long long)K * n * n * n;
  k_jacobian<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(dX[0], dX[1], dX[2], sJ, wJ, w, K, n, bad);
  return cudaGetLastError();
}

// per side node: master element e, local side s -> outward ntilde = sgn * Ja^l interpolated to the face
__global__ void k_faces(const double* __restrict__ Ja, const double* __restrict__ X, const int* __restrict__ sideMaster,
                        const double* __restrict__ lm, const double* __restrict__ lp, double* __restrict__ fgeo,
                        double* __restrict__ xbc, int S, int nBC, int n) {
  const int n2 = n * n, n3 = n2 * n;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)S * n2) return;
  const int side = idx / n2, pq = idx % n2;
  const int e = sideMaster[2 * side], s = sideMaster[2 * side + 1];
  const int l = s >> 1;
  const double sgn = (s & 1) ? 1.0 : -1.0;
  const double* lv = (s & 1) ? lp : lm;
  const int p = pq % n, q = pq / n;
  double nt[3] = {0, 0, 0}, xf[3] = {0, 0, 0};
  for (int a = 0; a < n; ++a) {
    const int vi = l == 0 ? a + n * (p + n * q) : (l == 1 ? p + n * (a + n * q) : p + n * (q + n * a));
    for (int d = 0; d < 3; ++d) {
      nt[d] += lv[a] * Ja[((long long)e * 9 + l * 3 + d) * n3 + vi];
      xf[d] += lv[a] * X[((long long)e * 3 + d) * n3 + vi];
    }
  }
  const double sa = sqrt(nt[0] * nt[0] + nt[1] * nt[1] + nt[2] * nt[2]);
  for (int d = 0; d < 3; ++d) fgeo[((long long)side * 4 + d) * n2 + pq] = sgn * nt[d] / sa;
  fgeo[((long long)side * 4 + 3) * n2 + pq] = sa;
  if (side < nBC)
    for (int d = 0; d < 3; ++d) xbc[((long long)side * 3 + d) * n2 + pq] = xf[d];
}

cudaError_t geom_faces(const double* Ja, const double* X, const int* sideMaster, const double* lm, const double* lp,
                       double* fgeo, double* xbc, int S, int nBC, int n, cudaStream_t st) {
  const long long tot = (long long)S * n * n;
  k_faces<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Ja, X, sideMaster, lm, lp, fgeo, xbc, S, nBC, n);
  return cudaGetLastError();
}

__global__ void k_f64_to_f32(const double* __restrict__ in, float* __restrict__ out, size_t count) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < count) out[idx] = (float)in[idx];
}

cudaError_t convert_f64_to_f32(const double* in, float* out, size_t count, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  k_f64_to_f32<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(in, out, count);
  return cudaGetLastError();
}

}  // namespace flexi
