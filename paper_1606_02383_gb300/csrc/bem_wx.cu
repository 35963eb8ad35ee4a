// bem_wx.cu -- the W- and X-list interactions of the adaptive octree.
//
// On an adaptive tree a leaf g and a finer box D below one of g's colleagues
// can be separated at D's scale (D does not touch g although D's parent does)
// without any pair of same-level boxes being in each other's V-list.  The
// FMM of Section 2.3 then takes the pair through one expansion:
//   M2P (W-list of g):  the multipole of D evaluated at g's targets,
//       z_i += sum_nm M~_D,nm h^_n(k|v|) Y_nm(v/|v|),   v = x_i - c_D;
//   P2L (X-list of D):  g's elements expanded about D's centre,
//       L~_D,nm += 4 pi i k sum_j sum_q [sigma_j F~_nm(v) - tau_j dF~_nm(v)/dn_j],
//       v = y_jq - c_D,  F~_nm(v) = h^_n(k|v|) conj(Y_nm(v/|v|)),
// with the conventions of the rest of the far field: orthonormal Y_nm
// without the Condon-Shortley phase, stored coefficients scaled by
// s_n = (k w)^n / (2n+1)!! of the expansion's level (M~ = M / s_n,
// L~ = L s_n), hence the scaled outgoing radial functions
// h^_n(x) = s_n h_n(x), which stay O(1) for every order.  The local
// expansion's form follows from Gegenbauer's theorem with source and target
// exchanged: G(x - y) = i k sum_nm h_n(k|y-c|) conj(Y_nm(y-c)) R_nm(x - c).
//
// The adjoint apply uses the plain transposes (the conjugations happen in its
// prologue and epilogue): M2P^T scatters target weights into the multipole
// adjoint of D, P2L^T gathers the local adjoint of D back to g's elements.
//
// Every radial and angular function is generated by recurrences on the fly:
//   h^_0 = h_0, h^_1 = (a/3) h_1, a = k w,
//   h^_{n+1} = a (2n+1) / ((2n+3) x) h^_n - a^2 / ((2n+1)(2n+3)) h^_{n-1},
// (from h_{n+1} = (2n+1)/x h_n - h_{n-1}; upward recurrence keeps the error
// relative to |h_n| since the outgoing solution dominates), with the
// derivative s_n h_n' = a/(2n+1) h^_{n-1} - (n+1)/x h^_n (n >= 1),
// s_0 h_0' = -(3/a) h^_1; and Y_nm(u) = W_n^m(u) (u_x + i u_y)^m for a unit
// vector u with the three-term recurrence of W in n.  The derivative along a
// direction d uses dual numbers: d|v| = u.d, du = (d - (u.d) u) / |v|.
#include <algorithm>
#include <cmath>
#include <vector>

#include "bem_common.cuh"
#include "bem_tree_walk.cuh"

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

#define WX_PMAX 40  // orders above this are rejected at setup (p_max <= 40)

template <typename R>
struct AV4x;
template <>
struct AV4x<float> {
  typedef float4 T;
};
template <>
struct AV4x<double> {
  typedef double4 T;
};

__device__ __forceinline__ void sc(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sc(double x, double* s, double* c) { sincos(x, s, c); }

// recurrence coefficients (filled at setup): for W_n^m, ca = sqrt((4n^2-1)/(n^2-m^2)),
// cb = sqrt(((n-1)^2-m^2)/(4(n-1)^2-1)); qmm = Ybar_mm, c1 = sqrt(2m+3); for h^_n,
// t1 = (2n+1)/(2n+3), t2 = 1/((2n+1)(2n+3)), t3 = 1/(2n+1)
#define WX_T (WX_PMAX + 2)
__constant__ float cf_ca[WX_T * WX_T], cf_cb[WX_T * WX_T], cf_q[WX_T], cf_c1[WX_T], cf_t1[WX_T], cf_t2[WX_T],
    cf_t3[WX_T];
__constant__ double cd_ca[WX_T * WX_T], cd_cb[WX_T * WX_T], cd_q[WX_T], cd_c1[WX_T], cd_t1[WX_T], cd_t2[WX_T],
    cd_t3[WX_T];
template <typename R>
struct WxTab;
template <>
struct WxTab<float> {
  __device__ static float ca(int i) { return cf_ca[i]; }
  __device__ static float cb(int i) { return cf_cb[i]; }
  __device__ static float q(int m) { return cf_q[m]; }
  __device__ static float c1(int m) { return cf_c1[m]; }
  __device__ static float t1(int n) { return cf_t1[n]; }
  __device__ static float t2(int n) { return cf_t2[n]; }
  __device__ static float t3(int n) { return cf_t3[n]; }
};
template <>
struct WxTab<double> {
  __device__ static double ca(int i) { return cd_ca[i]; }
  __device__ static double cb(int i) { return cd_cb[i]; }
  __device__ static double q(int m) { return cd_q[m]; }
  __device__ static double c1(int m) { return cd_c1[m]; }
  __device__ static double t1(int n) { return cd_t1[n]; }
  __device__ static double t2(int n) { return cd_t2[n]; }
  __device__ static double t3(int n) { return cd_t3[n]; }
};

// For NPT points v[q] (sharing the direction d of the derivative) and every
// (n, m), n <= p: F_nm = h^_n(k|v|) Y_nm(v/|v|) and, with DER, its
// derivative along d; fn(n, m, fr, fi, gr, gi) gets arrays over the points
// and is called for m = -n .. n.  The radial values h^_n (and derivatives)
// of every point are tabulated once per call in per-thread arrays; measured
// faster than rerunning the recurrence for every m in registers.
template <typename R, bool DER, int NPT, typename Fn>
__device__ __forceinline__ void outgoing_rows(int p, R k, R a, const R (&vx)[NPT], const R (&vy)[NPT],
                                              const R (&vz)[NPT], R dx, R dy, R dz, Fn&& fn) {
  typedef WxTab<R> T;
  R hr[NPT][WX_T], hi[NPT][WX_T], dhr[NPT][DER ? WX_T : 1], dhi[NPT][DER ? WX_T : 1];
  R ux[NPT], uy[NPT], uz[NPT], rd[NPT], dux[NPT], duy[NPT], duz[NPT];
  const R a2 = a * a, a3 = a / R(3);
#pragma unroll
  for (int q = 0; q < NPT; ++q) {
    const R r = sqrt(vx[q] * vx[q] + vy[q] * vy[q] + vz[q] * vz[q]);
    const R ir = R(1) / r;
    const R x = k * r, ix = ir / k;
    R sn, cs;
    sc(x, &sn, &cs);
    hr[q][0] = sn * ix;
    hi[q][0] = -cs * ix;
    hr[q][1] = a3 * ((-cs + sn * ix) * ix);  // h_1 = j_1 + i y_1
    hi[q][1] = a3 * ((-cs * ix - sn) * ix);
    const R aix = a * ix;
    for (int n = 1; n < p; ++n) {
      const R c1 = aix * T::t1(n), c2 = a2 * T::t2(n);
      hr[q][n + 1] = c1 * hr[q][n] - c2 * hr[q][n - 1];
      hi[q][n + 1] = c1 * hi[q][n] - c2 * hi[q][n - 1];
    }
    ux[q] = vx[q] * ir;
    uy[q] = vy[q] * ir;
    uz[q] = vz[q] * ir;
    rd[q] = dux[q] = duy[q] = duz[q] = 0;
    if constexpr (DER) {
      // d/dr of h^_n(k r)
      const R ka = k * (R(3) / a);
      dhr[q][0] = -ka * hr[q][1];
      dhi[q][0] = -ka * hi[q][1];
      for (int n = 1; n <= p; ++n) {
        const R c1 = a * T::t3(n), c2 = R(n + 1) * ix;
        dhr[q][n] = k * (c1 * hr[q][n - 1] - c2 * hr[q][n]);
        dhi[q][n] = k * (c1 * hi[q][n - 1] - c2 * hi[q][n]);
      }
      rd[q] = ux[q] * dx + uy[q] * dy + uz[q] * dz;
      dux[q] = (dx - rd[q] * ux[q]) * ir;
      duy[q] = (dy - rd[q] * uy[q]) * ir;
      duz[q] = (dz - rd[q] * uz[q]) * ir;
    }
  }
  // (u_x + i u_y)^m and its derivative
  R pr[NPT], pi[NPT], dpr[NPT], dpi[NPT];
#pragma unroll
  for (int q = 0; q < NPT; ++q) {
    pr[q] = 1;
    pi[q] = dpr[q] = dpi[q] = 0;
  }
  for (int m = 0; m <= p; ++m) {
    if (m > 0) {
#pragma unroll
      for (int q = 0; q < NPT; ++q) {
        const R npr = pr[q] * ux[q] - pi[q] * uy[q], npi = pr[q] * uy[q] + pi[q] * ux[q];
        if constexpr (DER) {
          const R ndr = dpr[q] * ux[q] - dpi[q] * uy[q] + pr[q] * dux[q] - pi[q] * duy[q];
          const R ndi = dpr[q] * uy[q] + dpi[q] * ux[q] + pr[q] * duy[q] + pi[q] * dux[q];
          dpr[q] = ndr;
          dpi[q] = ndi;
        }
        pr[q] = npr;
        pi[q] = npi;
      }
    }
    const R qmm = T::q(m);
    R w2[NPT], w1[NPT], dw2[NPT], dw1[NPT];
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
      w2[q] = dw2[q] = dw1[q] = 0;
      w1[q] = qmm;
    }
    for (int n = m; n <= p; ++n) {
      R fr[NPT], fi[NPT], gr[NPT], gi[NPT], cr[NPT], ci[NPT], er[NPT], ei[NPT];
      const R ca = (n >= m + 2) ? T::ca(n * WX_T + m) : R(0), cb = (n >= m + 2) ? T::cb(n * WX_T + m) : R(0);
      const R c1m = T::c1(m);
#pragma unroll
      for (int q = 0; q < NPT; ++q) {
        R w, dw = 0;
        if (n == m) {
          w = w1[q];
          dw = dw1[q];
        } else if (n == m + 1) {
          w = c1m * uz[q] * w1[q];
          if constexpr (DER) dw = c1m * (duz[q] * w1[q] + uz[q] * dw1[q]);
        } else {
          w = ca * (uz[q] * w1[q] - cb * w2[q]);
          if constexpr (DER) dw = ca * (duz[q] * w1[q] + uz[q] * dw1[q] - cb * dw2[q]);
        }
        if (n > m) {
          w2[q] = w1[q];
          w1[q] = w;
          dw2[q] = dw1[q];
          dw1[q] = dw;
        }
        // Y_nm = w (pr + i pi); Y_n,-m = conj(Y_nm)
        const R yr = w * pr[q], yi = w * pi[q];
        const R h_r = hr[q][n], h_i = hi[q][n];
        fr[q] = h_r * yr - h_i * yi;
        fi[q] = h_r * yi + h_i * yr;
        cr[q] = h_r * yr + h_i * yi;  // with conj(Y)
        ci[q] = -h_r * yi + h_i * yr;
        gr[q] = gi[q] = er[q] = ei[q] = 0;
        if constexpr (DER) {
          const R dyr = dw * pr[q] + w * dpr[q], dyi = dw * pi[q] + w * dpi[q];
          const R dh_r = rd[q] * dhr[q][n], dh_i = rd[q] * dhi[q][n];
          gr[q] = dh_r * yr - dh_i * yi + (h_r * dyr - h_i * dyi);
          gi[q] = dh_r * yi + dh_i * yr + (h_r * dyi + h_i * dyr);
          er[q] = dh_r * yr + dh_i * yi + (h_r * dyr + h_i * dyi);
          ei[q] = -dh_r * yi + dh_i * yr + (-h_r * dyi + h_i * dyr);
        }
      }
      fn(n, m, fr, fi, gr, gi);
      if (m > 0) fn(n, -m, cr, ci, er, ei);
    }
  }
}

__device__ __forceinline__ int wx_idx(int n, int m) { return n * n + n + m; }

// ------------------------------------------------------------------- M2P --
// One block per leaf with a W-list (x rhs); one thread per target of the
// leaf, looping over the leaf's W boxes.  Adds into the far sums.
template <typename R>
__global__ void k_m2p(const int* __restrict__ wleaves, const int* __restrict__ gl_start,
                      const int* __restrict__ gl_end, const int* __restrict__ w_ptr, const int* __restrict__ w_src,
                      const typename AV4x<R>::T* __restrict__ w_shift, LevTab lt, const int* __restrict__ lev_p,
                      const R* __restrict__ lev_a, R k, int64_t nt, const typename AV4x<R>::T* __restrict__ tgt,
                      const R* __restrict__ M, int64_t exp_stride, double* __restrict__ zfar) {
  const int g = wleaves[blockIdx.x];
  const int r = blockIdx.y;
  const R* Mr = M + 2 * (int64_t)r * exp_stride;
  for (int i = gl_start[g] + threadIdx.x; i < gl_end[g]; i += blockDim.x) {
    const typename AV4x<R>::T t = tgt[i];
    R sre = 0, sim = 0;
    for (int e = w_ptr[g]; e < w_ptr[g + 1]; ++e) {
      const int code = w_src[e], lvl = code >> 24, box = code & 0xFFFFFF;
      const typename AV4x<R>::T sh = w_shift[e];
      const R* Md = Mr + 2 * (lt.base[lvl] + (int64_t)box * lt.P[lvl]);
      const R vx[1] = {t.x + sh.x}, vy[1] = {t.y + sh.y}, vz[1] = {t.z + sh.z};
      outgoing_rows<R, false, 1>(lev_p[lvl], k, lev_a[lvl], vx, vy, vz, R(0), R(0), R(0),
                                 [&](int n, int m, const R* fr, const R* fi, const R*, const R*) {
                                   const int q = wx_idx(n, m);
                                   const R mr = Md[2 * q], mi = Md[2 * q + 1];
                                   sre += mr * fr[0] - mi * fi[0];
                                   sim += mr * fi[0] + mi * fr[0];
                                 });
    }
    double* z = zfar + 2 * ((int64_t)r * nt + i);
    z[0] += (double)sre;
    z[1] += (double)sim;
  }
}

// ------------------------------------------------------------------- P2L --
// One block per X pair (box B, leaf C) x rhs; one thread per element of C.
// The block sums its coefficients in shared memory, then adds them to B's
// local expansion (several pairs share a box: global atomics).
template <typename R>
__global__ void k_p2l(int npair, const int* __restrict__ xdst, const int* __restrict__ xsrc,
                      const typename AV4x<R>::T* __restrict__ xshift, int p, R a, R k, int64_t base,
                      const int* __restrict__ gl_start, const int* __restrict__ gl_end, int64_t nt,
                      const typename AV4x<R>::T* __restrict__ src, const typename AV4x<R>::T* __restrict__ dens,
                      R* __restrict__ L, int64_t exp_stride) {
  extern __shared__ __align__(16) unsigned char wx_smem[];
  R* acc = (R*)wx_smem;
  const int P = (p + 1) * (p + 1);
  const int pair = blockIdx.x, r = blockIdx.y;
  for (int q = threadIdx.x; q < 2 * P; q += blockDim.x) acc[q] = 0;
  __syncthreads();
  const int B = xdst[pair], C = xsrc[pair];
  const typename AV4x<R>::T sh = xshift[pair];
  const typename AV4x<R>::T* dr = dens + (int64_t)r * nt;
  for (int j = gl_start[C] + threadIdx.x; j < gl_end[C]; j += blockDim.x) {
    const typename AV4x<R>::T d = dr[j];
    const typename AV4x<R>::T q0 = src[3 * (int64_t)j], q1 = src[3 * (int64_t)j + 1], q2 = src[3 * (int64_t)j + 2];
    const R nx = q0.w, ny = q1.w, nz = q2.w;
    const R vx[3] = {q0.x + sh.x, q1.x + sh.x, q2.x + sh.x}, vy[3] = {q0.y + sh.y, q1.y + sh.y, q2.y + sh.y},
            vz[3] = {q0.z + sh.z, q1.z + sh.z, q2.z + sh.z};
    outgoing_rows<R, true, 3>(p, k, a, vx, vy, vz, nx, ny, nz,
                              [&](int n, int m, const R* fr, const R* fi, const R* gr, const R* gi) {
                                // the function of index (n, m) is F~_{n,-m} (conj(Y))
                                const int q = wx_idx(n, -m);
                                const R sfr = fr[0] + fr[1] + fr[2], sfi = fi[0] + fi[1] + fi[2];
                                const R sgr = gr[0] + gr[1] + gr[2], sgi = gi[0] + gi[1] + gi[2];
                                // sigma F - tau dF over the three points
                                atomicAdd(&acc[2 * q], d.x * sfr - d.y * sfi - (d.z * sgr - d.w * sgi));
                                atomicAdd(&acc[2 * q + 1], d.x * sfi + d.y * sfr - (d.z * sgi + d.w * sgr));
                              });
  }
  __syncthreads();
  // times 4 pi i k
  const R f = R(4.0 * BEM_PI) * k;
  R* Lb = L + 2 * ((int64_t)r * exp_stride + base + (int64_t)B * P);
  for (int q = threadIdx.x; q < P; q += blockDim.x) {
    const R ar = acc[2 * q], ai = acc[2 * q + 1];
    atomicAdd(&Lb[2 * q], -f * ai);
    atomicAdd(&Lb[2 * q + 1], f * ar);
  }
}

// ---------------------------------------------------------------- M2P^T --
// One block per (leaf with a W-list) x rhs: for each W box D of the leaf the
// threads (one per target) sum F_nm(x_i - c_D) h_i into shared memory, then
// add it to D's multipole adjoint.
template <typename R>
__global__ void k_m2p_t(const int* __restrict__ wleaves, const int* __restrict__ gl_start,
                        const int* __restrict__ gl_end, const int* __restrict__ w_ptr, const int* __restrict__ w_src,
                        const typename AV4x<R>::T* __restrict__ w_shift, LevTab lt, const int* __restrict__ lev_p,
                        const R* __restrict__ lev_a, R k, int64_t nt, const typename AV4x<R>::T* __restrict__ tgt,
                        const typename AV4x<R>::T* __restrict__ dens, R* __restrict__ Mu, int64_t exp_stride) {
  extern __shared__ __align__(16) unsigned char wx_smem[];
  R* acc = (R*)wx_smem;
  const int g = wleaves[blockIdx.x];
  const int r = blockIdx.y;
  const typename AV4x<R>::T* dr = dens + (int64_t)r * nt;
  for (int e = w_ptr[g]; e < w_ptr[g + 1]; ++e) {
    const int code = w_src[e], lvl = code >> 24, box = code & 0xFFFFFF;
    const int p = lev_p[lvl], P = (p + 1) * (p + 1);
    const typename AV4x<R>::T sh = w_shift[e];
    for (int q = threadIdx.x; q < 2 * P; q += blockDim.x) acc[q] = 0;
    __syncthreads();
    for (int i = gl_start[g] + threadIdx.x; i < gl_end[g]; i += blockDim.x) {
      const typename AV4x<R>::T t = tgt[i];
      const typename AV4x<R>::T hd = dr[i];
      const R vx[1] = {t.x + sh.x}, vy[1] = {t.y + sh.y}, vz[1] = {t.z + sh.z};
      outgoing_rows<R, false, 1>(p, k, lev_a[lvl], vx, vy, vz, R(0), R(0), R(0),
                                 [&](int n, int m, const R* fr, const R* fi, const R*, const R*) {
                                   const int q = wx_idx(n, m);
                                   atomicAdd(&acc[2 * q], fr[0] * hd.x - fi[0] * hd.y);
                                   atomicAdd(&acc[2 * q + 1], fr[0] * hd.y + fi[0] * hd.x);
                                 });
    }
    __syncthreads();
    R* Md = Mu + 2 * ((int64_t)r * exp_stride + lt.base[lvl] + (int64_t)box * lt.P[lvl]);
    for (int q = threadIdx.x; q < P; q += blockDim.x) {
      atomicAdd(&Md[2 * q], acc[2 * q]);
      atomicAdd(&Md[2 * q + 1], acc[2 * q + 1]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- P2L^T --
// One block per X pair x rhs; one thread per element of C:
// u_j += 4 pi i k sum_q sum_nm F~_nm Lam_nm, v_j += 4 pi i k sum_q sum_nm dF~_nm Lam_nm.
template <typename R>
__global__ void k_p2l_t(int npair, const int* __restrict__ xdst, const int* __restrict__ xsrc,
                        const typename AV4x<R>::T* __restrict__ xshift, int p, R a, R k, int64_t base,
                        const int* __restrict__ gl_start, const int* __restrict__ gl_end, int64_t nt,
                        const typename AV4x<R>::T* __restrict__ src, const R* __restrict__ Lam, int64_t exp_stride,
                        double4* __restrict__ uv) {
  const int P = (p + 1) * (p + 1);
  const int pair = blockIdx.x, r = blockIdx.y;
  const int B = xdst[pair], C = xsrc[pair];
  const typename AV4x<R>::T sh = xshift[pair];
  const R* Lb = Lam + 2 * ((int64_t)r * exp_stride + base + (int64_t)B * P);
  for (int j = gl_start[C] + threadIdx.x; j < gl_end[C]; j += blockDim.x) {
    const typename AV4x<R>::T q0 = src[3 * (int64_t)j], q1 = src[3 * (int64_t)j + 1], q2 = src[3 * (int64_t)j + 2];
    const R nx = q0.w, ny = q1.w, nz = q2.w;
    const R vx[3] = {q0.x + sh.x, q1.x + sh.x, q2.x + sh.x}, vy[3] = {q0.y + sh.y, q1.y + sh.y, q2.y + sh.y},
            vz[3] = {q0.z + sh.z, q1.z + sh.z, q2.z + sh.z};
    R ur = 0, ui = 0, vr = 0, vi = 0;
    outgoing_rows<R, true, 3>(p, k, a, vx, vy, vz, nx, ny, nz,
                              [&](int n, int m, const R* fr, const R* fi, const R* gr, const R* gi) {
                                const int q = wx_idx(n, -m);
                                const R lr = Lb[2 * q], li = Lb[2 * q + 1];
                                const R sfr = fr[0] + fr[1] + fr[2], sfi = fi[0] + fi[1] + fi[2];
                                const R sgr = gr[0] + gr[1] + gr[2], sgi = gi[0] + gi[1] + gi[2];
                                ur += sfr * lr - sfi * li;
                                ui += sfr * li + sfi * lr;
                                vr += sgr * lr - sgi * li;
                                vi += sgr * li + sgi * lr;
                              });
    // times 4 pi i k
    const R f = R(4.0 * BEM_PI) * k;
    double4* t = uv + (int64_t)r * nt + j;
    atomicAdd(&t->x, (double)(-f * ui));
    atomicAdd(&t->y, (double)(f * ur));
    atomicAdd(&t->z, (double)(-f * vi));
    atomicAdd(&t->w, (double)(f * vr));
  }
}

// --------------------------------------------------- M2P at field points --
// Forward-mode dual numbers v + d e (e^2 = 0): run through the M2P below with
// the point moved along a direction n (d of the coordinates = n), the value
// comes out with its derivative along n and the gradient with (Hess u) n.
template <typename R>
struct Dual {
  R v, d;
  __device__ __forceinline__ Dual() {}
  __device__ __forceinline__ Dual(R a) : v(a), d(R(0)) {}
  __device__ __forceinline__ Dual(R a, R b) : v(a), d(b) {}
  friend __device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
  friend __device__ __forceinline__ Dual operator+(Dual a, R b) { return Dual(a.v + b, a.d); }
  friend __device__ __forceinline__ Dual operator+(R a, Dual b) { return Dual(a + b.v, b.d); }
  friend __device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
  friend __device__ __forceinline__ Dual operator-(Dual a, R b) { return Dual(a.v - b, a.d); }
  friend __device__ __forceinline__ Dual operator-(R a, Dual b) { return Dual(a - b.v, -b.d); }
  friend __device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
  friend __device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.v * b.d + a.d * b.v); }
  friend __device__ __forceinline__ Dual operator*(Dual a, R b) { return Dual(a.v * b, a.d * b); }
  friend __device__ __forceinline__ Dual operator*(R a, Dual b) { return Dual(a * b.v, a * b.d); }
  friend __device__ __forceinline__ Dual operator/(Dual a, R b) { return Dual(a.v / b, a.d / b); }
  friend __device__ __forceinline__ Dual operator/(R a, Dual b) {
    const R q = a / b.v;
    return Dual(q, -q * b.d / b.v);
  }
  __device__ __forceinline__ Dual& operator+=(Dual b) {
    v += b.v;
    d += b.d;
    return *this;
  }
  friend __device__ __forceinline__ Dual sqrt(Dual a) {
    const R r = sqrt(a.v);
    return Dual(r, a.d / (R(2) * r));
  }
};
template <typename R>
__device__ __forceinline__ void sc(Dual<R> x, Dual<R>* s, Dual<R>* c) {
  R sn, cs;
  sc(x.v, &sn, &cs);
  *s = Dual<R>(sn, cs * x.d);
  *c = Dual<R>(cs, -sn * x.d);
}

// The multipole of one far box evaluated at one point (the off-surface walk,
// bem_tree_walk.cuh), for NR right-hand sides at once: the same h^_n, Y_nm
// recurrences as outgoing_rows, with the pair (n, m), (n, -m) folded into
// Z = M~_nm Y_nm + M~_n,-m conj(Y_nm), so that
//   u += sum_n h^_n Z_n,
//   grad u += (v/|v|) sum_n h^_n'(r) Z_n + sum_n h^_n grad Z_n,
// grad Z taking grad Y_nm = grad(W_n^m(u_z)) (u_x + i u_y)^m + W_n^m grad (u_x + i u_y)^m
// with du_a/dv_c = (delta_ac - u_a u_c) / |v| (the chain rule through u = v / |v|).
// D is the number type of everything that depends on the point: R, or Dual<R>.
template <typename R, typename D, bool GRAD, int NR>
__device__ __forceinline__ void m2p_point_t(int p, R k, R a, D vx, D vy, D vz, const R* const (&Md)[NR],
                                            D (&val)[NR][2], D (&grd)[NR][3][2]) {
  typedef WxTab<R> T;
  D hr[WX_T], hi[WX_T], dhr[GRAD ? WX_T : 1], dhi[GRAD ? WX_T : 1];
  const D r = sqrt(vx * vx + vy * vy + vz * vz);
  const D ir = R(1) / r;
  const D x = k * r, ix = ir / k;
  D sn, cs;
  sc(x, &sn, &cs);
  const R a2 = a * a, a3 = a / R(3);
  hr[0] = sn * ix;
  hi[0] = -cs * ix;
  hr[1] = a3 * ((-cs + sn * ix) * ix);
  hi[1] = a3 * ((-cs * ix - sn) * ix);
  const D aix = a * ix;
  for (int n = 1; n < p; ++n) {
    const D c1 = aix * T::t1(n);
    const R c2 = a2 * T::t2(n);
    hr[n + 1] = c1 * hr[n] - c2 * hr[n - 1];
    hi[n + 1] = c1 * hi[n] - c2 * hi[n - 1];
  }
  const D u[3] = {vx * ir, vy * ir, vz * ir};
  D dux[3], duy[3], duz[3];
  if constexpr (GRAD) {
    const R ka = k * (R(3) / a);
    dhr[0] = -ka * hr[1];
    dhi[0] = -ka * hi[1];
    for (int n = 1; n <= p; ++n) {
      const R c1 = a * T::t3(n);
      const D c2 = R(n + 1) * ix;
      dhr[n] = k * (c1 * hr[n - 1] - c2 * hr[n]);
      dhi[n] = k * (c1 * hi[n - 1] - c2 * hi[n]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      dux[c] = ((c == 0 ? R(1) : R(0)) - u[0] * u[c]) * ir;
      duy[c] = ((c == 1 ? R(1) : R(0)) - u[1] * u[c]) * ir;
      duz[c] = ((c == 2 ? R(1) : R(0)) - u[2] * u[c]) * ir;
    }
  }
  D Ar[NR], Ai[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) Ar[q] = Ai[q] = D(R(0));
  D pr = D(R(1)), pi = D(R(0)), dpr[3], dpi[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) dpr[c] = dpi[c] = D(R(0));
  for (int m = 0; m <= p; ++m) {
    if (m > 0) {
      const D npr = pr * u[0] - pi * u[1], npi = pr * u[1] + pi * u[0];
      if constexpr (GRAD) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const D ndr = dpr[c] * u[0] - dpi[c] * u[1] + pr * dux[c] - pi * duy[c];
          const D ndi = dpr[c] * u[1] + dpi[c] * u[0] + pr * duy[c] + pi * dux[c];
          dpr[c] = ndr;
          dpi[c] = ndi;
        }
      }
      pr = npr;
      pi = npi;
    }
    D w1 = D(T::q(m)), w2 = D(R(0)), dw1[3], dw2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) dw1[c] = dw2[c] = D(R(0));
    const R c1m = T::c1(m);
    for (int n = m; n <= p; ++n) {
      D w, dw[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) dw[c] = D(R(0));
      if (n == m) {
        w = w1;
      } else if (n == m + 1) {
        w = (c1m * u[2]) * w1;
        if constexpr (GRAD)
#pragma unroll
          for (int c = 0; c < 3; ++c) dw[c] = c1m * (duz[c] * w1 + u[2] * dw1[c]);
      } else {
        const R ca = T::ca(n * WX_T + m), cb = T::cb(n * WX_T + m);
        w = ca * (u[2] * w1 - cb * w2);
        if constexpr (GRAD)
#pragma unroll
          for (int c = 0; c < 3; ++c) dw[c] = ca * (duz[c] * w1 + u[2] * dw1[c] - cb * dw2[c]);
      }
      if (n > m) {
        w2 = w1;
        w1 = w;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          dw2[c] = dw1[c];
          dw1[c] = dw[c];
        }
      }
      const D yr = w * pr, yi = w * pi;
      const D h_r = hr[n], h_i = hi[n];
      const int qp = wx_idx(n, m), qm = wx_idx(n, -m);
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        const R mpr = Md[q][2 * qp], mpi = Md[q][2 * qp + 1];
        // Z = M+ Y + M- conj(Y)
        D zr = mpr * yr - mpi * yi, zi = mpr * yi + mpi * yr;
        R mmr = 0, mmi = 0;
        if (m > 0) {
          mmr = Md[q][2 * qm];
          mmi = Md[q][2 * qm + 1];
          zr = zr + (mmr * yr + mmi * yi);
          zi = zi + (-mmr * yi + mmi * yr);
        }
        val[q][0] += h_r * zr - h_i * zi;
        val[q][1] += h_r * zi + h_i * zr;
        if constexpr (GRAD) {
          Ar[q] += dhr[n] * zr - dhi[n] * zi;
          Ai[q] += dhr[n] * zi + dhi[n] * zr;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const D dyr = dw[c] * pr + w * dpr[c], dyi = dw[c] * pi + w * dpi[c];
            const D gzr = mpr * dyr - mpi * dyi + (mmr * dyr + mmi * dyi);
            const D gzi = mpr * dyi + mpi * dyr + (-mmr * dyi + mmi * dyr);
            grd[q][c][0] += h_r * gzr - h_i * gzi;
            grd[q][c][1] += h_r * gzi + h_i * gzr;
          }
        }
      }
    }
  }
  if constexpr (GRAD) {
#pragma unroll
    for (int q = 0; q < NR; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        grd[q][c][0] += u[c] * Ar[q];
        grd[q][c][1] += u[c] * Ai[q];
      }
  }
}
template <typename R, bool GRAD, int NR>
__device__ __forceinline__ void m2p_point(int p, R k, R a, R vx, R vy, R vz, const R* const (&Md)[NR],
                                          R (&val)[NR][2], R (&grd)[NR][3][2]) {
  m2p_point_t<R, R, GRAD, NR>(p, k, a, vx, vy, vz, Md, val, grd);
}

// Teams of `team` consecutive lanes (a power of two, at most 32) per field
// point (in the walk's order): the lanes of a team walk the tree together,
// each keeping a list of the far boxes it takes (the c-th far box goes to lane
// c mod team; beyond WALK_OWN of them a lane evaluates at once), evaluate
// their lists side by side after the walk, then sum their parts over the
// team.  team = 1 for dense point sets;
// larger teams keep the GPU full when the points are few (the vertex
// gradient's on-surface points).  Lanes past the last point walk nothing but
// take part in the team sums.
template <int NV>
__device__ __forceinline__ void team_sum(float (&v)[NV], int team) {
  for (int o = team >> 1; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
}
template <int NV>
__device__ __forceinline__ void team_sum(double (&v)[NV], int team) {
  for (int o = team >> 1; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
}

// The multipoles of the point's far boxes.  Writes acc[r][i][c] (FP64
// complex), c over the components of the mode (0: u; 1: grad u; 2: u, grad u),
// and nearflag[i]: whether the point's walk has near leaves.
template <typename R, int MODE, int NR>
__global__ void __launch_bounds__(128) k_evf_far(int64_t np, int r0, int team, WalkTree wt,
                                                 const double* __restrict__ pts, const int* __restrict__ tcs,
                                                 LevTab lt, const int* __restrict__ lev_p,
                                                 const R* __restrict__ lev_a, R k, const R* __restrict__ M,
                                                 int64_t exp_stride, double* __restrict__ acc,
                                                 int* __restrict__ nearflag) {
  constexpr bool GRAD = MODE != 0;
  constexpr int NC = MODE == 0 ? 1 : (MODE == 1 ? 3 : 4);
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i = gt / team;
  const int tl = (int)(gt & (team - 1));
  const bool live = i < np;
  bool near = false;
  R val[NR][2], grd[NR][3][2];
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    val[q][0] = val[q][1] = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) grd[q][c][0] = grd[q][c][1] = 0;
  }
  if (live) {
    const double X[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
    const int t[3] = {tcs[3 * i], tcs[3 * i + 1], tcs[3 * i + 2]};
    auto m2p = [&](int l, int b) {
      const double* c = wt.lv[l].centre + 3 * b;
      const R vx = (R)(X[0] - c[0]), vy = (R)(X[1] - c[1]), vz = (R)(X[2] - c[2]);
      const R* Md[NR];
#pragma unroll
      for (int q = 0; q < NR; ++q)
        Md[q] = M + 2 * ((int64_t)(r0 + q) * exp_stride + lt.base[l] + (int64_t)b * lt.P[l]);
      m2p_point<R, GRAD, NR>(lev_p[l], k, lev_a[l], vx, vy, vz, Md, val, grd);
    };
    int own[WALK_OWN], no = 0, cnt = 0;
    tree_walk(wt, t, [&](int kind, int l, int b) {
      if (kind != 0) {
        near = true;
        return;
      }
      if (team == 1) {
        m2p(l, b);
        return;
      }
      if ((cnt++ & (team - 1)) != tl) return;
      if (no < WALK_OWN)
        own[no++] = (l << 24) | b;
      else
        m2p(l, b);
    });
    for (int u = 0; u < no; ++u) m2p(own[u] >> 24, own[u] & 0xFFFFFF);
  }
  if (team > 1) {
    R v[NR * 8];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      v[8 * q] = val[q][0];
      v[8 * q + 1] = val[q][1];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        v[8 * q + 2 + 2 * c] = grd[q][c][0];
        v[8 * q + 3 + 2 * c] = grd[q][c][1];
      }
    }
    team_sum(v, team);
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      val[q][0] = v[8 * q];
      val[q][1] = v[8 * q + 1];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        grd[q][c][0] = v[8 * q + 2 + 2 * c];
        grd[q][c][1] = v[8 * q + 3 + 2 * c];
      }
    }
  }
  if (!live || tl != 0) return;
  if (r0 == 0) nearflag[i] = near ? 1 : 0;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    double* o = acc + 2 * (((int64_t)(r0 + q) * np + i) * NC);
    int c0 = 0;
    if (MODE != 1) {
      o[0] = (double)val[q][0];
      o[1] = (double)val[q][1];
      c0 = 1;
    }
    if (GRAD)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        o[2 * (c0 + c)] = (double)grd[q][c][0];
        o[2 * (c0 + c) + 1] = (double)grd[q][c][1];
      }
  }
}

// The vertex gradient's source side, far boxes: a team of lanes per walk point
// (as in k_evf_far), a quadrature point of element j = perm[i] / 3.  The
// multipoles are those of the point charges conj(g_i) at the centroids, so the
// walk sums psi(y) = sum_i conj(g_i) G(y - x_i); with the point moved along
// the normal n_j as a dual number it returns psi, n.grad psi, grad psi and
// (Hess psi) n.  Writes acc[r][i][0..7] (FP64 complex) = psi, grad psi (3),
// n.grad psi, (Hess psi) n (3).
template <typename R, int NR>
__global__ void __launch_bounds__(128) k_gvf_far(int64_t np, int r0, int team, WalkTree wt,
                                                 const double* __restrict__ pts, const int* __restrict__ tcs,
                                                 const int* __restrict__ perm, const double* __restrict__ nrm,
                                                 LevTab lt, const int* __restrict__ lev_p,
                                                 const R* __restrict__ lev_a, R k, const R* __restrict__ M,
                                                 int64_t exp_stride, double* __restrict__ acc) {
  typedef Dual<R> D;
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i = gt / team;
  const int tl = (int)(gt & (team - 1));
  const bool live = i < np;
  D val[NR][2], grd[NR][3][2];
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    val[q][0] = val[q][1] = D(R(0));
#pragma unroll
    for (int c = 0; c < 3; ++c) grd[q][c][0] = grd[q][c][1] = D(R(0));
  }
  if (live) {
    const double X[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
    const int t[3] = {tcs[3 * i], tcs[3 * i + 1], tcs[3 * i + 2]};
    const int64_t j = perm[i] / 3;
    const R n[3] = {(R)nrm[3 * j], (R)nrm[3 * j + 1], (R)nrm[3 * j + 2]};
    auto m2p = [&](int l, int b) {
      const double* c = wt.lv[l].centre + 3 * b;
      const D vx((R)(X[0] - c[0]), n[0]), vy((R)(X[1] - c[1]), n[1]), vz((R)(X[2] - c[2]), n[2]);
      const R* Md[NR];
#pragma unroll
      for (int q = 0; q < NR; ++q)
        Md[q] = M + 2 * ((int64_t)(r0 + q) * exp_stride + lt.base[l] + (int64_t)b * lt.P[l]);
      m2p_point_t<R, D, true, NR>(lev_p[l], k, lev_a[l], vx, vy, vz, Md, val, grd);
    };
    int own[WALK_OWN], no = 0, cnt = 0;
    tree_walk(wt, t, [&](int kind, int l, int b) {
      if (kind != 0) return;
      if ((cnt++ & (team - 1)) != tl) return;
      if (no < WALK_OWN)
        own[no++] = (l << 24) | b;
      else
        m2p(l, b);
    });
    for (int u = 0; u < no; ++u) m2p(own[u] >> 24, own[u] & 0xFFFFFF);
  }
  // component order of acc: psi, grad psi (3), n.grad psi, (Hess psi) n (3)
  R v[NR * 16];
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    v[16 * q] = val[q][0].v;
    v[16 * q + 1] = val[q][1].v;
    v[16 * q + 8] = val[q][0].d;
    v[16 * q + 9] = val[q][1].d;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v[16 * q + 2 + 2 * c] = grd[q][c][0].v;
      v[16 * q + 3 + 2 * c] = grd[q][c][1].v;
      v[16 * q + 10 + 2 * c] = grd[q][c][0].d;
      v[16 * q + 11 + 2 * c] = grd[q][c][1].d;
    }
  }
  team_sum(v, team);
  if (!live || tl != 0) return;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    double* o = acc + 16 * ((int64_t)(r0 + q) * np + i);
#pragma unroll
    for (int c = 0; c < 16; ++c) o[c] = (double)v[16 * q + c];
  }
}

// -------------------------------------------------------------------- host --
// orders and k w_l of every level in the operator's precision (setup)
int bem_build_wx_tables(bem_handle* h, cudaStream_t s) {
  int hp[BEM_MAXLEV + 1];
  double ha[BEM_MAXLEV + 1];
  float haf[BEM_MAXLEV + 1];
  for (int l = 0; l <= BEM_MAXLEV; ++l) {
    const bool has = l >= 2 && l <= h->L;
    hp[l] = has ? h->lev[l].p : 0;
    ha[l] = has ? h->k * h->lev[l].w : 1.0;
    haf[l] = (float)ha[l];
    if (has && h->lev[l].p > WX_PMAX) return bem_fail(BEM_ERR_UNSUPPORTED, "expansion order above 40");
  }
  {
    static double ca[WX_T * WX_T], cb[WX_T * WX_T], q[WX_T], c1[WX_T], t1[WX_T], t2[WX_T], t3[WX_T];
    static float fca[WX_T * WX_T], fcb[WX_T * WX_T], fq[WX_T], fc1[WX_T], ft1[WX_T], ft2[WX_T], ft3[WX_T];
    double qmm = 0.28209479177387814347;
    for (int m = 0; m < WX_T; ++m) {
      if (m > 0) qmm *= std::sqrt((2.0 * m + 1.0) / (2.0 * m));
      q[m] = qmm;
      c1[m] = std::sqrt(2.0 * m + 3.0);
      t1[m] = (2.0 * m + 1.0) / (2.0 * m + 3.0);
      t2[m] = 1.0 / ((2.0 * m + 1.0) * (2.0 * m + 3.0));
      t3[m] = 1.0 / (2.0 * m + 1.0);
    }
    for (int n = 0; n < WX_T; ++n)
      for (int m = 0; m < WX_T; ++m) {
        const bool ok = n >= m + 2;
        ca[n * WX_T + m] = ok ? std::sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m)) : 0.0;
        cb[n * WX_T + m] =
            ok ? std::sqrt(((double)(n - 1) * (n - 1) - (double)m * m) / (4.0 * (n - 1) * (n - 1) - 1.0)) : 0.0;
      }
    for (int i = 0; i < WX_T * WX_T; ++i) {
      fca[i] = (float)ca[i];
      fcb[i] = (float)cb[i];
    }
    for (int i = 0; i < WX_T; ++i) {
      fq[i] = (float)q[i];
      fc1[i] = (float)c1[i];
      ft1[i] = (float)t1[i];
      ft2[i] = (float)t2[i];
      ft3[i] = (float)t3[i];
    }
    BEM_CUDA(cudaMemcpyToSymbolAsync(cd_ca, ca, sizeof(ca), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyToSymbolAsync(cd_cb, cb, sizeof(cb), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyToSymbolAsync(cd_q, q, sizeof(q), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyToSymbolAsync(cd_c1, c1, sizeof(c1), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyToSymbolAsync(cd_t1, t1, sizeof(t1), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyToSymbolAsync(cd_t2, t2, sizeof(t2), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyToSymbolAsync(cd_t3, t3, sizeof(t3), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyToSymbolAsync(cf_ca, fca, sizeof(fca), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyToSymbolAsync(cf_cb, fcb, sizeof(fcb), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyToSymbolAsync(cf_q, fq, sizeof(fq), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyToSymbolAsync(cf_c1, fc1, sizeof(fc1), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyToSymbolAsync(cf_t1, ft1, sizeof(ft1), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyToSymbolAsync(cf_t2, ft2, sizeof(ft2), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyToSymbolAsync(cf_t3, ft3, sizeof(ft3), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaStreamSynchronize(s));  // the static host arrays are reused by later handles
  }
  BEM_TRY(bem_alloc(h, &h->wx_p, BEM_MAXLEV + 1));
  double* a;
  BEM_TRY(bem_alloc(h, &a, BEM_MAXLEV + 1));
  h->wx_a = a;
  BEM_CUDA(cudaMemcpyAsync(h->wx_p, hp, sizeof(hp), cudaMemcpyHostToDevice, s));
  if (bem_is_fp64(h))
    BEM_CUDA(cudaMemcpyAsync(h->wx_a, ha, sizeof(ha), cudaMemcpyHostToDevice, s));
  else
    BEM_CUDA(cudaMemcpyAsync(h->wx_a, haf, sizeof(haf), cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaStreamSynchronize(s));
  return BEM_OK;
}

template <typename R>
static int run_m2p(bem_handle* h, int nrhs, const void* M, double* zfar, cudaStream_t s, int* launches) {
  if (h->n_w_leaves == 0 || !bem_is_fmm(h) || h->L < 2) return BEM_OK;
  const int* dp = h->wx_p;
  const void* da = h->wx_a;
  typedef typename AV4x<R>::T V4;
  const V4* tgt = (const V4*)(sizeof(R) == 4 ? (const void*)h->tgt32 : (const void*)h->tgt64);
  const V4* wsh = (const V4*)(sizeof(R) == 4 ? (const void*)h->w_shift32 : (const void*)h->w_shift64);
  k_m2p<R><<<dim3(h->n_w_leaves, nrhs), 64, 0, s>>>(h->w_leaves, h->gl_start, h->gl_end, h->w_ptr, h->w_src, wsh,
                                                    bem_levtab(h), dp, (const R*)da, (R)h->k, h->nt, tgt, (const R*)M,
                                                    h->exp_total, zfar);
  BEM_CUDA(cudaGetLastError());
  ++*launches;
  return BEM_OK;
}

template <typename R>
static int run_p2l(bem_handle* h, int nrhs, const void* dens, void* Lexp, cudaStream_t s, int* launches) {
  if (!bem_is_fmm(h) || h->L < 2) return BEM_OK;
  typedef typename AV4x<R>::T V4;
  const V4* src = (const V4*)(sizeof(R) == 4 ? (const void*)h->src32 : (const void*)h->src64);
  for (int l = 2; l <= h->L; ++l) {
    if (h->x_n[l] == 0) continue;
    const LevelInfo& lv = h->lev[l];
    const V4* xsh = (const V4*)(sizeof(R) == 4 ? (const void*)h->x_shift32[l] : (const void*)h->x_shift64[l]);
    const size_t smem = 2 * sizeof(R) * (size_t)lv.P;
    if (smem > 48 * 1024)
      BEM_CUDA(cudaFuncSetAttribute(k_p2l<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_p2l<R><<<dim3(h->x_n[l], nrhs), 64, smem, s>>>(h->x_n[l], h->x_dst[l], h->x_src[l], xsh, lv.p,
                                                     (R)(h->k * lv.w), (R)h->k, lv.exp_base, h->gl_start, h->gl_end,
                                                     h->nt, src, (const V4*)dens, (R*)Lexp, h->exp_total);
    BEM_CUDA(cudaGetLastError());
    ++*launches;
  }
  return BEM_OK;
}

template <typename R>
static int run_m2p_t(bem_handle* h, int nrhs, const void* dens, void* Mu, cudaStream_t s, int* launches) {
  if (h->n_w_leaves == 0 || !bem_is_fmm(h) || h->L < 2) return BEM_OK;
  const int* dp = h->wx_p;
  const void* da = h->wx_a;
  typedef typename AV4x<R>::T V4;
  const V4* tgt = (const V4*)(sizeof(R) == 4 ? (const void*)h->tgt32 : (const void*)h->tgt64);
  const V4* wsh = (const V4*)(sizeof(R) == 4 ? (const void*)h->w_shift32 : (const void*)h->w_shift64);
  int Pmax = 0;
  for (int l = 2; l <= h->L; ++l) Pmax = std::max(Pmax, h->lev[l].P);
  const size_t smem = 2 * sizeof(R) * (size_t)Pmax;
  if (smem > 48 * 1024)
    BEM_CUDA(cudaFuncSetAttribute(k_m2p_t<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_m2p_t<R><<<dim3(h->n_w_leaves, nrhs), 64, smem, s>>>(h->w_leaves, h->gl_start, h->gl_end, h->w_ptr, h->w_src,
                                                         wsh, bem_levtab(h), dp, (const R*)da, (R)h->k, h->nt, tgt,
                                                         (const V4*)dens, (R*)Mu, h->exp_total);
  BEM_CUDA(cudaGetLastError());
  ++*launches;
  return BEM_OK;
}

template <typename R>
static int run_p2l_t(bem_handle* h, int nrhs, const void* Lam, double4* uv, cudaStream_t s, int* launches) {
  if (!bem_is_fmm(h) || h->L < 2) return BEM_OK;
  typedef typename AV4x<R>::T V4;
  const V4* src = (const V4*)(sizeof(R) == 4 ? (const void*)h->src32 : (const void*)h->src64);
  for (int l = 2; l <= h->L; ++l) {
    if (h->x_n[l] == 0) continue;
    const LevelInfo& lv = h->lev[l];
    const V4* xsh = (const V4*)(sizeof(R) == 4 ? (const void*)h->x_shift32[l] : (const void*)h->x_shift64[l]);
    k_p2l_t<R><<<dim3(h->x_n[l], nrhs), 64, 0, s>>>(h->x_n[l], h->x_dst[l], h->x_src[l], xsh, lv.p,
                                                    (R)(h->k * lv.w), (R)h->k, lv.exp_base, h->gl_start, h->gl_end,
                                                    h->nt, src, (const R*)Lam, h->exp_total, uv);
    BEM_CUDA(cudaGetLastError());
    ++*launches;
  }
  return BEM_OK;
}

int bem_run_m2p(bem_handle* h, int nrhs, const void* M, double* zfar, cudaStream_t s, int* launches) {
  return bem_is_fp64(h) ? run_m2p<double>(h, nrhs, M, zfar, s, launches)
                        : run_m2p<float>(h, nrhs, M, zfar, s, launches);
}
int bem_run_p2l(bem_handle* h, int nrhs, const void* dens, void* Lexp, cudaStream_t s, int* launches) {
  return bem_is_fp64(h) ? run_p2l<double>(h, nrhs, dens, Lexp, s, launches)
                        : run_p2l<float>(h, nrhs, dens, Lexp, s, launches);
}
int bem_run_m2p_t(bem_handle* h, int nrhs, const void* dens, void* Mu, cudaStream_t s, int* launches) {
  return bem_is_fp64(h) ? run_m2p_t<double>(h, nrhs, dens, Mu, s, launches)
                        : run_m2p_t<float>(h, nrhs, dens, Mu, s, launches);
}
int bem_run_p2l_t(bem_handle* h, int nrhs, const void* Lam, double4* uv, cudaStream_t s, int* launches) {
  return bem_is_fp64(h) ? run_p2l_t<double>(h, nrhs, Lam, uv, s, launches)
                        : run_p2l_t<float>(h, nrhs, Lam, uv, s, launches);
}

template <typename R, int MODE>
static int evf_far_impl(bem_handle* h, const WalkTree& wt, int nrhs, int64_t np, const double* pts, const int* tcs,
                        double* acc, int* nearflag, int team, cudaStream_t s) {
  const LevTab lt = bem_levtab(h);
  const unsigned g = nblk(np * team, 128);
  for (int r0 = 0; r0 < nrhs;) {
    const int rem = nrhs - r0;
#define EVF_FAR(NRV)                                                                                       \
  k_evf_far<R, MODE, NRV><<<g, 128, 0, s>>>(np, r0, team, wt, pts, tcs, lt, h->wx_p, (const R*)h->wx_a,   \
                                            (R)h->k, (const R*)h->Mexp, h->exp_total, acc, nearflag);      \
  r0 += NRV;
    if (rem >= 4) {
      EVF_FAR(4)
    } else if (rem >= 2) {
      EVF_FAR(2)
    } else {
      EVF_FAR(1)
    }
#undef EVF_FAR
    BEM_CUDA(cudaGetLastError());
  }
  return BEM_OK;
}

int bem_evf_far(bem_handle* h, const WalkTree& wt, int nrhs, int mode, int64_t np, const double* pts,
                const int* tcs, double* acc, int* nearflag, int team, cudaStream_t s) {
  if (team < 1 || team > 32 || (team & (team - 1))) return bem_fail(BEM_ERR_INVALID_ARG, "bad walk team size");
  const bool f64 = bem_is_fp64(h);
  if (mode == 0) return f64 ? evf_far_impl<double, 0>(h, wt, nrhs, np, pts, tcs, acc, nearflag, team, s)
                            : evf_far_impl<float, 0>(h, wt, nrhs, np, pts, tcs, acc, nearflag, team, s);
  if (mode == 1) return f64 ? evf_far_impl<double, 1>(h, wt, nrhs, np, pts, tcs, acc, nearflag, team, s)
                            : evf_far_impl<float, 1>(h, wt, nrhs, np, pts, tcs, acc, nearflag, team, s);
  return f64 ? evf_far_impl<double, 2>(h, wt, nrhs, np, pts, tcs, acc, nearflag, team, s)
             : evf_far_impl<float, 2>(h, wt, nrhs, np, pts, tcs, acc, nearflag, team, s);
}

template <typename R>
static int gvf_far_impl(bem_handle* h, const WalkTree& wt, int nrhs, int64_t np, const double* pts, const int* tcs,
                        const int* perm, int team, double* acc, cudaStream_t s) {
  const LevTab lt = bem_levtab(h);
  const unsigned g = nblk(np * team, 128);
  for (int r0 = 0; r0 < nrhs;) {
    const int rem = nrhs - r0;
#define GVF_FAR(NRV)                                                                                          \
  k_gvf_far<R, NRV><<<g, 128, 0, s>>>(np, r0, team, wt, pts, tcs, perm, h->nrm, lt, h->wx_p, (const R*)h->wx_a, \
                                      (R)h->k, (const R*)h->Mexp, h->exp_total, acc);                          \
  r0 += NRV;
    if (rem >= 4) {
      GVF_FAR(4)
    } else if (rem >= 2) {
      GVF_FAR(2)
    } else {
      GVF_FAR(1)
    }
#undef GVF_FAR
    BEM_CUDA(cudaGetLastError());
  }
  return BEM_OK;
}

int bem_gvf_far(bem_handle* h, const WalkTree& wt, int nrhs, int64_t np, const double* pts, const int* tcs,
                const int* perm, int team, double* acc, cudaStream_t s) {
  if (team < 1 || team > 32 || (team & (team - 1))) return bem_fail(BEM_ERR_INVALID_ARG, "bad walk team size");
  return bem_is_fp64(h) ? gvf_far_impl<double>(h, wt, nrhs, np, pts, tcs, perm, team, acc, s)
                        : gvf_far_impl<float>(h, wt, nrhs, np, pts, tcs, perm, team, acc, s);
}
