// Akima spline motion model (Sec. II-B.1) and its vector-Jacobian product,
// in FP64 (it is part of the geometry, next to Eq. 1).
//
// Each of the six motion parameters p is an Akima spline through node
// values y_i = nodes[i][p], i < n, at knots x_i = i (V-1)/(n-1) (first knot
// at view 0, last at view V-1); theta[j][p] is the spline at x = j.
//   secants      m_i = (y_{i+1} - y_i) / h,  h = (V-1)/(n-1)
//   end secants  linear extrapolation of the secant sequence, two per end
//   node slopes  t_i = (w1 m_{i-1} + w2 m_i) / (w1 + w2) with
//                w1 = |m_{i+1} - m_i|, w2 = |m_{i-1} - m_{i-2}|, and the mean
//                of m_{i-1}, m_i where w1 + w2 = 0
//   pieces       cubic Hermite of (y_i, t_i), (y_{i+1}, t_{i+1}) on [x_i, x_{i+1}]
// One CTA per parameter; the secant array s[k] = m_{k-2} (k < n+3) and the
// slopes live in shared memory.  The VJP runs the same steps backwards
// (reverse mode), in gather form so that every sum has a fixed order.
#include "bp_internal.cuh"

namespace bpk {

namespace {

constexpr int SPT = 256;

__device__ __forceinline__ double knot(int i, int n, int V) {
  return i == n - 1 ? (double)(V - 1) : (double)i * ((double)(V - 1) / (double)(n - 1));
}

// Secants (with the extrapolated ends) and node slopes of parameter p.
__device__ void akima_setup(int n, int V, const double* __restrict__ nodes, int p, double* s,
                            double* t) {
  for (int i = threadIdx.x; i + 1 < n; i += blockDim.x)
    s[i + 2] = (nodes[(i + 1) * 6 + p] - nodes[i * 6 + p]) / (knot(i + 1, n, V) - knot(i, n, V));
  __syncthreads();
  if (threadIdx.x == 0) {
    s[1] = 2.0 * s[2] - s[3];
    s[0] = 2.0 * s[1] - s[2];
    s[n + 1] = 2.0 * s[n] - s[n - 1];
    s[n + 2] = 2.0 * s[n + 1] - s[n];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double w1 = fabs(s[i + 3] - s[i + 2]), w2 = fabs(s[i + 1] - s[i]);
    const double den = w1 + w2;
    t[i] = den == 0.0 ? 0.5 * (s[i + 1] + s[i + 2]) : (w1 * s[i + 1] + w2 * s[i + 2]) / den;
  }
  __syncthreads();
}

// Interval of view j: the largest i <= n-2 with x_i <= j.
__device__ __forceinline__ int interval(int j, int n, int V) {
  const long long i = (long long)j * (n - 1) / (V - 1);
  return (int)min(i, (long long)(n - 2));
}

__global__ void __launch_bounds__(SPT) akima_eval_kernel(int n, int V,
                                                         const double* __restrict__ nodes,
                                                         double* __restrict__ theta) {
  extern __shared__ double sm[];
  double* s = sm;           // n + 3
  double* t = sm + n + 3;   // n
  const int p = blockIdx.x;
  akima_setup(n, V, nodes, p, s, t);
  for (int j = threadIdx.x; j < V; j += blockDim.x) {
    const int i = interval(j, n, V);
    const double xi = knot(i, n, V), h = knot(i + 1, n, V) - xi, e = (double)j - xi;
    const double m = s[i + 2];
    const double c = (3.0 * m - 2.0 * t[i] - t[i + 1]) / h;
    const double d = (t[i] + t[i + 1] - 2.0 * m) / (h * h);
    theta[j * 6 + p] = nodes[i * 6 + p] + t[i] * e + (c * e * e + d * e * e * e);
  }
}

__global__ void __launch_bounds__(SPT) akima_vjp_kernel(int n, int V,
                                                        const double* __restrict__ nodes,
                                                        const double* __restrict__ g,
                                                        double* __restrict__ dnodes) {
  extern __shared__ double sm[];
  double* s = sm;               // n + 3  secants
  double* t = s + n + 3;        // n      slopes
  double* A = t + n;            // n - 1  per interval: sum of g            (-> y_i)
  double* B = A + n - 1;        // n - 1  sum of g dp/dt_i                  (-> t_i)
  double* C = B + n - 1;        // n - 1  sum of g dp/dt_{i+1}              (-> t_{i+1})
  double* D = C + n - 1;        // n - 1  sum of g dp/dm_i                  (-> m_i)
  double* tb = D + n - 1;       // n      adjoint of t
  double* sb = tb + n;          // n + 3  adjoint of s
  const int p = blockIdx.x;
  akima_setup(n, V, nodes, p, s, t);
  // per interval, its views in order
  for (int i = threadIdx.x; i < n - 1; i += blockDim.x) {
    const double xi = knot(i, n, V), h = knot(i + 1, n, V) - xi;
    // views of interval i: j in [ceil(x_i), next interval's first view)
    int j0 = (int)(((long long)i * (V - 1) + (n - 2)) / (n - 1));
    int j1 = i == n - 2 ? V : (int)(((long long)(i + 1) * (V - 1) + (n - 2)) / (n - 1));
    double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
    for (int j = j0; j < j1; ++j) {
      const double gj = g[j * 6 + p], e = (double)j - xi, q = e / h;
      a += gj;
      b += gj * (e * (1.0 - q) * (1.0 - q));
      c += gj * (e * q * (q - 1.0));
      d += gj * (e * q * (3.0 - 2.0 * q));
    }
    A[i] = a;
    B[i] = b;
    C[i] = c;
    D[i] = d;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    tb[i] = (i < n - 1 ? B[i] : 0.0) + (i > 0 ? C[i - 1] : 0.0);
  __syncthreads();
  // t_i -> s[i .. i+3], gathered per s index k from i = k-3 .. k
  for (int k = threadIdx.x; k < n + 3; k += blockDim.x) {
    double acc = (k >= 2 && k - 2 < n - 1) ? D[k - 2] : 0.0;
    for (int i = max(0, k - 3); i <= min(k, n - 1); ++i) {
      const int o = k - i;
      const double w1 = fabs(s[i + 3] - s[i + 2]), w2 = fabs(s[i + 1] - s[i]);
      const double den = w1 + w2;
      double dt;
      if (den == 0.0) {
        dt = (o == 1 || o == 2) ? 0.5 : 0.0;
      } else {
        const double ti = t[i];
        const double sg1 = (s[i + 3] > s[i + 2]) ? 1.0 : (s[i + 3] < s[i + 2] ? -1.0 : 0.0);
        const double sg2 = (s[i + 1] > s[i]) ? 1.0 : (s[i + 1] < s[i] ? -1.0 : 0.0);
        const double f1 = (s[i + 1] - ti) / den, f2 = (s[i + 2] - ti) / den;  // dt/dw1, dt/dw2
        if (o == 0) dt = -sg2 * f2;
        else if (o == 1) dt = w1 / den + sg2 * f2;
        else if (o == 2) dt = w2 / den - sg1 * f1;
        else dt = sg1 * f1;
      }
      acc += tb[i] * dt;
    }
    sb[k] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // extrapolated ends, in reverse order of their definition
    sb[1] += 2.0 * sb[0];
    sb[2] -= sb[0];
    sb[2] += 2.0 * sb[1];
    sb[3] -= sb[1];
    sb[n + 1] += 2.0 * sb[n + 2];
    sb[n] -= sb[n + 2];
    sb[n] += 2.0 * sb[n + 1];
    sb[n - 1] -= sb[n + 1];
  }
  __syncthreads();
  // secants -> node values: s[i+2] = (y_{i+1} - y_i) / h_i
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double acc = k < n - 1 ? A[k] : 0.0;
    if (k >= 1) acc += sb[k + 1] / (knot(k, n, V) - knot(k - 1, n, V));
    if (k <= n - 2) acc -= sb[k + 2] / (knot(k + 1, n, V) - knot(k, n, V));
    dnodes[k * 6 + p] = acc;
  }
}

}  // namespace

size_t akima_smem_bytes(int n, bool vjp) {
  return sizeof(double) * (size_t)(vjp ? (n + 3) * 2 + n * 2 + 4 * (n - 1) : (n + 3) + n);
}

cudaError_t launch_akima_eval(int n, int V, const double* nodes, double* theta, cudaStream_t st) {
  akima_eval_kernel<<<6, SPT, akima_smem_bytes(n, false), st>>>(n, V, nodes, theta);
  return cudaGetLastError();
}

cudaError_t launch_akima_vjp(int n, int V, const double* nodes, const double* g, double* dnodes,
                             cudaStream_t st) {
  akima_vjp_kernel<<<6, SPT, akima_smem_bytes(n, true), st>>>(n, V, nodes, g, dnodes);
  return cudaGetLastError();
}

}  // namespace bpk
