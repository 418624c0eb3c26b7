// Point-to-plane ICP in SE(3) and Sim(3) with the frame-to-keyframe photometric term
// (Sec. 5, 5.1-5.3; Sec. 6 for Sim(3); Sec. 8 outlier thresholds).
//
// One launch = one Gauss-Newton iteration: a persistent grid (2 CTAs per SM) walks the
// pixels of the current pyramid level grid-stride, forms each pixel's point-to-plane row
// (and photometric row) in registers, accumulates w J J^T (upper triangle), w J r, w r^2
// and the row counts in FP32, reduces them by warp shuffles and across warps in a fixed
// order, and stores one partial per CTA. The last CTA to finish (atomic ticket) adds the
// partials in FP64 in a fixed order - so the result is bitwise reproducible - then one
// warp solves H xi = -g by FP64 Cholesky and applies dT <- exp(xi) dT on the device.
#include <math.h>

#include <cooperative_groups.h>

#include "internal.h"

namespace dtsdf {

constexpr int ICP_THREADS = ICP_CTA_THREADS;

// ------------------------------------------------------------- pyramid ----
__global__ void k_extract_depth(const float4* __restrict__ P, int n, float* __restrict__ d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float4 p = P[i];
    d[i] = p.w > 0 ? p.z : 0.0f;
  }
}

// Intensity I = (0.299 R + 0.587 G + 0.114 B) / 255 is kept through the pyramid as the integer
// sum S = 299 R + 587 G + 114 B over the level's 4^l source pixels (at most 255000 * 4^3 < 2^24,
// so every sum and difference of sums is exact in FP32); a level's intensity is S / (255000 4^l)
// and its central-difference gradient (S(+1) - S(-1)) / (2 * 255000 4^l), each correctly rounded.
__global__ void k_intensity(const uint8_t* __restrict__ rgb, int n, float* __restrict__ S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) S[i] = (float)(299 * (int)rgb[3 * i] + 587 * (int)rgb[3 * i + 1] + 114 * (int)rgb[3 * i + 2]);
}

// 2x2 mean of the valid depth children in the order (0,0), (1,0), (0,1), (1,1); 2x2 sum of the
// intensity sums.
__global__ void k_down(const float* __restrict__ din, const float* __restrict__ Sin, int Win, int Wout, int Hout,
                       float* __restrict__ dout, float* __restrict__ Sout) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= Wout || v >= Hout) return;
  const int i00 = (2 * v) * Win + 2 * u;
  const float c[4] = {din[i00], din[i00 + 1], din[i00 + Win], din[i00 + Win + 1]};
  float s = 0.0f;
  int n = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (c[q] > 0.0f) {
      s = radd(s, c[q]);
      ++n;
    }
  dout[v * Wout + u] = n ? rdiv(s, (float)n) : 0.0f;
  if (Sin) Sout[v * Wout + u] = (Sin[i00] + Sin[i00 + 1]) + (Sin[i00 + Win] + Sin[i00 + Win + 1]);
}

__global__ void k_down_intensity(const float* __restrict__ Sin, int Win, int Wout, int Hout, float* __restrict__ Sout) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= Wout || v >= Hout) return;
  const int i00 = (2 * v) * Win + 2 * u;
  Sout[v * Wout + u] = (Sin[i00] + Sin[i00 + 1]) + (Sin[i00 + Win] + Sin[i00 + Win + 1]);
}

// intensity sums of a level -> intensities (in place)
__global__ void k_norm_intensity(float* __restrict__ S, int n, float c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) S[i] = rdiv(S[i], c);
}

// Keyframe level: (I, dI/du, dI/dv, 0) from the intensity sums, central differences / 2, zero on
// the border.
__global__ void k_kf_grad(const float* __restrict__ S, int W, int H, float c, float4* __restrict__ out) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= W || v >= H) return;
  const int i = v * W + u;
  const float gx = (u >= 1 && u < W - 1) ? rdiv(S[i + 1] - S[i - 1], 2.0f * c) : 0.0f;
  const float gy = (v >= 1 && v < H - 1) ? rdiv(S[i + W] - S[i - W], 2.0f * c) : 0.0f;
  out[i] = make_float4(rdiv(S[i], c), gx, gy, 0.0f);
}

// ------------------------------------------------------------- FP64 math --
__device__ void mat4_mul(const double* A, const double* B, double* C) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0;
      for (int k = 0; k < 4; ++k) s += A[4 * i + k] * B[4 * k + j];
      C[4 * i + j] = s;
    }
}

// Exponential of the 4x4 generator [[omega^ + sigma I, nu], [0, 0]]:
//   upper block e^sigma exp(omega^) (Rodrigues), translation V nu with
//   V = A I + B omega^ + C omega^2, A = int_0^1 e^{s sigma} ds,
//   B = (1/th) int_0^1 e^{s sigma} sin(s th) ds, C = (1/th^2) (A - int_0^1 e^{s sigma} cos(s th) ds),
// with series where th or sigma vanish.
// The transcendental values sin(th), cos(th), e^sigma and e^sigma - 1 (th = |omega|) are
// passed in, so that a warp can evaluate them in parallel lanes.
// Evaluated by one warp, as the solve uses it: every lane forms the scalar
// coefficients (identical values; reciprocals instead of repeated divisions: GB300's FP64 rate is
// low, so the dependent FP64 chain is the solve's latency), lanes 0-11 one entry each of the top
// 3x4 block of T, lanes 12-15 the last row. T: shared or global, written by lanes 0-15.
__device__ void exp_sim3_warp(const double* xi, int dim, double sin_th, double cos_th, double es, double em1,
                              double* T, int lane) {
  const double nu0 = xi[0], nu1 = xi[1], nu2 = xi[2];
  const double w0 = xi[3], w1 = xi[4], w2 = xi[5];
  const double sg = dim == 7 ? xi[6] : 0.0;
  const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
  const double th = sqrt(th2);
  const bool small = th < 1e-4;
  const double inv_th = small ? 0.0 : 1.0 / th;
  const double inv_th2 = inv_th * inv_th;
  double a, b;  // sin(th)/th, (1 - cos th)/th^2
  if (small) {
    a = 1.0 - th2 * (1.0 / 6.0) + th2 * th2 * (1.0 / 120.0);
    b = 0.5 - th2 * (1.0 / 24.0) + th2 * th2 * (1.0 / 720.0);
  } else {
    a = sin_th * inv_th;
    b = (1.0 - cos_th) * inv_th2;
  }
  const double A = sg != 0.0 ? em1 / sg : 1.0;
  double B, C;
  if (small) {
    // expansions of the integrals in th (exact in sigma), leading orders
    double I1, I2, I3;  // int s e^{s sg}, int s^2 e^{s sg} / 2, int s^3 e^{s sg} / 6 over [0, 1]
    if (fabs(sg) < 1e-2) {
      // sum_n sg^n / (n! (n + k)) with k = 2, 3, 4
      double t = 1.0;
      I1 = I2 = I3 = 0.0;
      for (int n = 0; n < 6; ++n) {
        I1 += t / (n + 2);
        I2 += t / (2.0 * (n + 3));
        I3 += t / (6.0 * (n + 4));
        t *= sg / (n + 1);
      }
    } else {
      const double s2 = sg * sg, s3 = s2 * sg, s4 = s3 * sg;
      I1 = ((sg - 1.0) * es + 1.0) / s2;
      I2 = ((s2 - 2.0 * sg + 2.0) * es - 2.0) / (2.0 * s3);
      I3 = ((s3 - 3.0 * s2 + 6.0 * sg - 6.0) * es + 6.0) / (6.0 * s4);
    }
    // sin(s th)/th = s - th^2 s^3/6 + ..., (1 - cos(s th))/th^2 = s^2/2 - ...
    B = I1 - th2 * I3;
    C = I2;
  } else {
    const double inv_D = sg != 0.0 ? 1.0 / (sg * sg + th2) : inv_th2;
    const double Is = (es * (sg * sin_th - th * cos_th) + th) * inv_D;
    const double Ic = (es * (sg * cos_th + th * sin_th) - sg) * inv_D;
    B = Is * inv_th;
    C = (A - Ic) * inv_th2;
  }
  if (lane >= 16) return;
  if (lane >= 12) {
    T[lane] = lane == 15 ? 1.0 : 0.0;
    return;
  }
  const int i = lane >> 2, j = lane & 3;
  // row i of omega^ and of omega^2 (omega^ = [[0,-w2,w1],[w2,0,-w0],[-w1,w0,0]])
  const double r0 = i == 0 ? 0.0 : (i == 1 ? w2 : -w1);
  const double r1 = i == 0 ? -w2 : (i == 1 ? 0.0 : w0);
  const double r2 = i == 0 ? w1 : (i == 1 ? -w0 : 0.0);
  const double q0 = r1 * w2 - r2 * w1;  // (omega^2)_{i,0} = row_i . column 0 = (0, w2, -w1)
  const double q1 = -r0 * w2 + r2 * w0; // column 1 = (-w2, 0, w0)
  const double q2 = r0 * w1 - r1 * w0;  // column 2 = (w1, -w0, 0)
  if (j < 3) {
    const double wij = j == 0 ? r0 : (j == 1 ? r1 : r2);
    const double qij = j == 0 ? q0 : (j == 1 ? q1 : q2);
    T[4 * i + j] = es * ((i == j ? 1.0 : 0.0) + a * wij + b * qij);
  } else {
    const double V0 = A * (i == 0) + B * r0 + C * q0;
    const double V1 = A * (i == 1) + B * r1 + C * q1;
    const double V2 = A * (i == 2) + B * r2 + C * q2;
    T[4 * i + 3] = V0 * nu0 + V1 * nu1 + V2 * nu2;
  }
}

__global__ void k_exp(int dim, const double* xi, double* T) {
  const int lane = threadIdx.x & 31;
  const double th = sqrt(xi[3] * xi[3] + xi[4] * xi[4] + xi[5] * xi[5]);
  const double sg = dim == 7 ? xi[6] : 0.0;
  double s_th, c_th;
  sincos(th, &s_th, &c_th);
  exp_sim3_warp(xi, dim, s_th, c_th, exp(sg), expm1(sg), T, lane);
}

// Solve and update of one Gauss-Newton iteration from the FP64 sums (layout of Acc<DIM>:
// upper triangle of H, g, E, geometric rows, photometric rows) for the leading dsolve
// unknowns (dsolve = DIM, or 6 for an SE(3) problem accumulated with DIM = 7): FP64
// Cholesky of H xi = -g (Eq. ICP_solution; a pivot below 1e-10 max diag(H), or fewer than
// min_rows rows, is a degenerate system), then pose <- exp(xi) pose (Eq. deltaT_update).
// Records the iteration in *st. Returns true when the level is finished (converged:
// ||xi|| < stop_norm, or degenerate: pose unchanged).
// Run by the 32 lanes of one warp (every lane calls it with the same sums; FP64
// throughout). The FP64 units are few, so what bounds this step is the length of its
// dependent chains: the Cholesky factor is formed column by column with the trailing update
// spread over the lanes, the triangular solves column-oriented, the sine, cosine and
// exponentials of the exponential map in separate lanes and the pose product one entry per
// lane. Every lane returns the same level decision.
// With lm (Levenberg-Marquardt, Sec. 7, with Madsen's damping update): the first evaluation of a
// level is accepted and sets mu = 1e-3 max diag(H), nu = 2; a later one is accepted when the gain
// ratio rho = (E_acc - E) / (predicted decrease) is positive (mu <- mu max(1/3, 1 - (2 rho - 1)^3),
// nu <- 2), otherwise the pose returns to the accepted one (mu <- mu nu, nu <- 2 nu). The step
// solves (H_acc + mu I) xi = -g_acc, its predicted decrease of E is xi^T H_acc xi + 2 mu xi^T xi
// (E(xi) ~ E + 2 g^T xi + xi^T H xi without the factor 2), and pose <- exp(xi) pose_acc.
template <int DIM>
__device__ bool icp_solve_update_warp(const double* sum, int dsolve, double* pose, dtsdf_icp_stats* st,
                                      int min_rows, double stop_norm, LmState* lm = nullptr) {
  constexpr int NH = DIM * (DIM + 1) / 2;
  constexpr int N = NH + DIM + 3;
  __shared__ double sL[7][8];
  __shared__ double sInv[8];  // 1 / L_jj
  __shared__ double sb[8];
  __shared__ double sgv[8];
  __shared__ double sE[16];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int D = dsolve;
  for (int k = lane; k < NH; k += 32) {
    int i = 0, r = k;  // entry k of the row-major upper triangle
    while (r >= DIM - i) {
      r -= DIM - i;
      ++i;
    }
    sL[i][i + r] = sL[i + r][i] = sum[k];
  }
  __syncwarp();
  for (int k = lane; k < 49; k += 32) {
    const int i = k / 7, j = k % 7;
    st->H[k] = (i < D && j < D) ? sL[i][j] : 0.0;
  }
  if (lane < 7) {
    st->g[lane] = lane < D ? sum[NH + lane] : 0.0;
    st->xi[lane] = 0.0;
  }
  const int64_t rows_photo = (int64_t)sum[N - 1];
  const int64_t rows = (int64_t)sum[N - 2] + rows_photo;
  if (lane == 0) {
    st->error = sum[NH + DIM];
    st->rows_photo = rows_photo;
    st->rows = rows;
    st->dim = D;
    st->iterations += 1;
    st->step_norm = 0.0;
    st->converged = 0;
  }
  double dmax = lane < D ? sL[lane][lane] : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(FULL, dmax, o));
  if (lane < D) sgv[lane] = sum[NH + lane];
  bool ok = rows >= min_rows && dmax > 0.0;
  double mu = 0.0;
  if (lm && ok) {
    int accept = 1;
    if (lane == 0) {
      const double E = sum[NH + DIM];
      if (!lm->have) {
        lm->mu = 1e-3 * dmax;
        lm->nu = 2.0;
      } else {
        const double rho = (lm->E - E) / lm->pred;
        accept = rho > 0.0;
        if (accept) {
          const double c = 2.0 * rho - 1.0;
          lm->mu *= fmax(1.0 / 3.0, 1.0 - c * c * c);
          lm->nu = 2.0;
        } else {
          lm->mu *= lm->nu;
          lm->nu *= 2.0;
        }
      }
      if (accept) {
        lm->E = E;
        lm->have = 1;
      }
    }
    accept = __shfl_sync(FULL, accept, 0);
    __syncwarp();
    mu = lm->mu;
    // the accepted system and pose: this evaluation's, or the stored ones
    for (int k = lane; k < 49; k += 32) {
      const int i = k / 7, j = k % 7;
      if (i < D && j < D) {
        if (accept)
          lm->H[k] = sL[i][j];
        else
          sL[i][j] = lm->H[k];
      }
    }
    if (lane < D) {
      if (accept)
        lm->g[lane] = sgv[lane];
      else
        sgv[lane] = lm->g[lane];
    }
    if (lane < 16) {
      if (accept)
        lm->pose[lane] = pose[lane];
      else
        pose[lane] = lm->pose[lane];
    }
    __syncwarp();
    if (lane < D) sL[lane][lane] += mu;
    __syncwarp();
    dmax = lane < D ? sL[lane][lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(FULL, dmax, o));
  }
  // Cholesky H = L L^T (lower triangle of sL), a pivot below 1e-10 max diag(H): degenerate
  for (int j = 0; j < D && ok; ++j) {
    const double s = sL[j][j];
    if (!(s > 1e-10 * dmax)) {
      ok = false;
      break;
    }
    const double inv = rsqrt(s), ljj = s * inv;  // one FP64 chain for the pivot and its reciprocal
    __syncwarp();
    if (lane == j) {
      sL[j][j] = ljj;
      sInv[j] = inv;
    }
    if (lane > j && lane < D) sL[lane][j] = sL[lane][j] * inv;
    __syncwarp();
    const int m = D - 1 - j;  // trailing lower triangle, rows and columns j + 1 .. D - 1
    for (int p = lane; p < m * (m + 1) / 2; p += 32) {
      int ii = 0, kk = p;
      while (kk > ii) {
        kk -= ii + 1;
        ++ii;
      }
      const int i = j + 1 + ii, k = j + 1 + kk;
      sL[i][k] -= sL[i][j] * sL[k][j];
    }
    __syncwarp();
  }
  if (!ok) {
    if (lane == 0) st->status = DTSDF_ERR_DEGENERATE;
    __syncwarp();
    return true;
  }
  // L y = -g, then L^T xi = y (column-oriented; sb holds the right-hand side, then xi)
  if (lane < D) sb[lane] = -sgv[lane];
  __syncwarp();
  for (int i = 0; i < D; ++i) {
    const double y = sb[i] * sInv[i];
    __syncwarp();
    if (lane == i) sb[i] = y;
    if (lane > i && lane < D) sb[lane] -= sL[lane][i] * y;
    __syncwarp();
  }
  for (int i = D - 1; i >= 0; --i) {
    const double x = sb[i] * sInv[i];
    __syncwarp();
    if (lane == i) sb[i] = x;
    if (lane < i) sb[lane] -= sL[i][lane] * x;
    __syncwarp();
  }
  double xi[7];
  double nrm = 0.0;
  for (int i = 0; i < 7; ++i) {
    xi[i] = i < D ? sb[i] : 0.0;
    nrm += xi[i] * xi[i];
  }
  nrm = sqrt(nrm);
  if (lm && lane == 0) {  // predicted decrease of E for the next gain ratio
    double q = 0.0;
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) q += xi[i] * lm->H[7 * i + j] * xi[j];
    lm->pred = q + 2.0 * mu * (nrm * nrm);
  }
  // exponential map: sin and cos in lane 1, e^sigma and e^sigma - 1 in lanes 3 and 4 (Sim(3)
  // only; 1 and 0 for SE(3)), then the entries of exp(xi) over lanes 0-15
  const double th = sqrt(xi[3] * xi[3] + xi[4] * xi[4] + xi[5] * xi[5]);
  const double sg = D == 7 ? xi[6] : 0.0;
  double fs = 0.0, fc = 1.0, fe = 1.0, fm = 0.0;
  // sin and cos are used only beyond the series range of exp_sim3_warp (th >= 1e-4)
  if (lane == 1 && !(th < 1e-4)) sincos(th, &fs, &fc);
  if (D == 7 && lane == 3) fe = exp(sg);
  if (D == 7 && lane == 4) fm = expm1(sg);
  const double s_th = __shfl_sync(FULL, fs, 1), c_th = __shfl_sync(FULL, fc, 1);
  const double es = __shfl_sync(FULL, fe, 3), em1 = __shfl_sync(FULL, fm, 4);
  exp_sim3_warp(xi, D, s_th, c_th, es, em1, sE, lane);
  __syncwarp();
  double t = 0.0;
  if (lane < 16) {
    const int i = lane >> 2, j = lane & 3;
    for (int k = 0; k < 4; ++k) t += sE[4 * i + k] * pose[4 * k + j];
  }
  __syncwarp();
  if (lane < 16) pose[lane] = t;
  if (lane < D) st->xi[lane] = xi[lane];
  if (lane == 0) {
    st->status = 0;
    st->step_norm = nrm;
    st->converged = nrm < stop_norm;
  }
  __syncwarp();
  return nrm < stop_norm;
}

// ---------------------------------------------------------- reduction -----
struct IcpArgs {
  // current level
  const float* depth;
  const float* inten;
  int W, H;
  float fx, fy, cx, cy;
  // reference render (full resolution)
  const float4* ref;  // normal xyz, w = depth
  int rW, rH;
  float rfx, rfy, rcx, rcy;
  float eps, zmin;
  // photometric
  const float4* kf;  // (I, gx, gy, 0) at this level
  int kW, kH;
  float kfx, kfy, kcx, kcy;
  float Rrs[9], trs[3];
  const double* Trs_dev;  // render -> keyframe camera in device memory (overrides Rrs/trs)
  float thr, lambda;
  // state
  double* pose;
  LmState* lm;
  float* partials;
  uint32_t* ticket;
  int32_t* stop;
  dtsdf_icp_stats* stats;
  int min_rows;
  double stop_norm;
};

// Per-thread FP32 accumulators of one Gauss-Newton system; KAHAN adds a compensation term
// per sum (Kahan summation over the pixels a thread visits).
template <int DIM, bool KAHAN>
struct Acc {
  static constexpr int NH = DIM * (DIM + 1) / 2;
  static constexpr int N = NH + DIM + 3;  // H upper, g, E, rows_geo, rows_photo
  float v[N];
  float c[KAHAN ? N : 1];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = 0.f;
#pragma unroll
    for (int i = 0; i < (KAHAN ? N : 1); ++i) c[i] = 0.f;
  }
  __device__ __forceinline__ void add(int i, float x) {
    if (KAHAN) {
      const float y = x - c[i];
      const float t = v[i] + y;
      c[i] = (t - v[i]) - y;
      v[i] = t;
    } else {
      v[i] += x;
    }
  }
  __device__ __forceinline__ void row(const float J[DIM], float r, float w) {
    int k = 0;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      const float wj = w * J[i];
#pragma unroll
      for (int j = i; j < DIM; ++j) add(k++, wj * J[j]);
      add(NH + i, wj * r);
    }
    add(NH + DIM, w * r * r);
  }
  // compensated value of sum i
  __device__ __forceinline__ float total(int i) const { return KAHAN ? v[i] - c[i] : v[i]; }
};

// Point-to-plane row of one current-frame pixel (Eq. geometric_ICP, Eq. ICP_geometric_dx,
// weight of Eq. ICP_weight): back-project depth z at (u, v) with the level intrinsics, move
// it by the estimate x = p + ((A p) + t) (A = sR - I), associate it with the nearest pixel of
// the full-resolution render (normals with the depth in w) and, for an inlier
// (||q - x|| <= eps), add w J J^T, w J r, w r^2 and the row count. The scale column of
// Sim(3) is filled when `scale` is set (DIM = 7), else left zero. Returns the moved point
// and the depth weight for the photometric row.
template <int DIM, bool KAHAN>
__device__ __forceinline__ void geo_row(Acc<DIM, KAHAN>& acc, float z, int u, int v, float fx, float fy, float cx,
                                        float cy, const float Am[9], const float tv[3], const float4* __restrict__ ref,
                                        int rW, int rH, float rfx, float rfy, float rcx, float rcy, float eps2,
                                        float zmin, bool scale, float& x0, float& x1, float& x2, float& wz) {
  using A = Acc<DIM, KAHAN>;
  const float P0 = rmul(z, rdiv(rsub((float)u, cx), fx));
  const float P1 = rmul(z, rdiv(rsub((float)v, cy), fy));
  const float P2 = z;
  const float d0 = radd(rdot3(Am[0], Am[1], Am[2], P0, P1, P2), tv[0]);
  const float d1 = radd(rdot3(Am[3], Am[4], Am[5], P0, P1, P2), tv[1]);
  const float d2 = radd(rdot3(Am[6], Am[7], Am[8], P0, P1, P2), tv[2]);
  x0 = radd(P0, d0);
  x1 = radd(P1, d1);
  x2 = radd(P2, d2);
  const float zw = z + 1.0f - zmin;
  wz = 1.0f / (zw * zw);  // Eq. ICP_weight
  if (!(x2 > 0.0f)) return;
  // projective association into the full-resolution render, nearest pixel
  const float uf = radd(rmul(rdiv(x0, x2), rfx), rcx);
  const float vf = radd(rmul(rdiv(x1, x2), rfy), rcy);
  const float ur = floorf(radd(uf, 0.5f)), vr = floorf(radd(vf, 0.5f));
  if (!(ur >= 0.0f && vr >= 0.0f && ur < (float)rW && vr < (float)rH)) return;
  const float4 nq = __ldg(ref + (int)vr * rW + (int)ur);
  const float dr = nq.w;
  if (!(dr > 0.0f)) return;
  const float q0 = rmul(dr, rdiv(rsub(ur, rcx), rfx));
  const float q1 = rmul(dr, rdiv(rsub(vr, rcy), rfy));
  const float q2 = dr;
  const float e0 = rsub(q0, x0), e1 = rsub(q1, x1), e2 = rsub(q2, x2);
  if (!(rdot3(e0, e1, e2, e0, e1, e2) <= eps2)) return;
  // r = <q - x, n> evaluated as <(q - p) - delta, n> (no cancellation of metre-sized terms)
  const float r = ((q0 - P0) - d0) * nq.x + ((q1 - P1) - d1) * nq.y + ((q2 - P2) - d2) * nq.z;
  float J[DIM];
  J[0] = -nq.x;
  J[1] = -nq.y;
  J[2] = -nq.z;
  J[3] = -(x1 * nq.z - x2 * nq.y);
  J[4] = -(x2 * nq.x - x0 * nq.z);
  J[5] = -(x0 * nq.y - x1 * nq.x);
  if (DIM == 7) J[DIM - 1] = scale ? -(nq.x * x0 + nq.y * x1 + nq.z * x2) : 0.0f;
  acc.row(J, r, wz);
  acc.v[A::N - 2] += 1.0f;  // a count, exact in FP32 below 2^24
}

template <int DIM, bool PHOTO, bool KAHAN>
__global__ void __launch_bounds__(ICP_THREADS) k_icp(IcpArgs a) {
  using A = Acc<DIM, KAHAN>;
  __shared__ float s_red[ICP_THREADS / 32][A::N];
  __shared__ double s_sum[A::N];
  __shared__ int s_last;
  __shared__ float s_pose[24];
  if (*((volatile int32_t*)a.stop)) return;  // level finished (converged or degenerate)

  // current estimate: x = p + ((A p) + t), A = sR - I (single precision, rounded); the FP64 pose
  // is rounded once per CTA (the FP64 rate is low), then read by every thread
  if (threadIdx.x < 12) {
    const int i = threadIdx.x >> 2, j = threadIdx.x & 3;
    const double v = a.pose[4 * i + j];
    s_pose[threadIdx.x] = (float)(j == 3 ? v : v - (i == j ? 1.0 : 0.0));
  } else if (PHOTO && a.Trs_dev && threadIdx.x < 24) {
    const int k = threadIdx.x - 12, i = k >> 2, j = k & 3;
    s_pose[threadIdx.x] = __double2float_rn(a.Trs_dev[4 * i + j]);
  }
  __syncthreads();
  float Am[9], tv[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) Am[3 * i + j] = s_pose[4 * i + j];
    tv[i] = s_pose[4 * i + 3];
  }
  if (PHOTO && a.Trs_dev) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int j = 0; j < 3; ++j) a.Rrs[3 * i + j] = s_pose[12 + 4 * i + j];
      a.trs[i] = s_pose[12 + 4 * i + 3];
    }
  }
  A acc;
  acc.zero();
  const int n = a.W * a.H;
  const float eps2 = rmul(a.eps, a.eps);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const float z = __ldg(a.depth + p);
    if (!(z > 0.0f)) continue;
    const int u = p % a.W, v = p / a.W;
    float x0, x1, x2, wz;
    geo_row<DIM, KAHAN>(acc, z, u, v, a.fx, a.fy, a.cx, a.cy, Am, tv, a.ref, a.rW, a.rH, a.rfx, a.rfy, a.rcx, a.rcy,
                        eps2, a.zmin, true, x0, x1, x2, wz);
    if (PHOTO) {
      // frame-to-keyframe photometric row (Eq. keyframe_icp), y = T_rs x
      const float y0 = radd(rdot3(a.Rrs[0], a.Rrs[1], a.Rrs[2], x0, x1, x2), a.trs[0]);
      const float y1 = radd(rdot3(a.Rrs[3], a.Rrs[4], a.Rrs[5], x0, x1, x2), a.trs[1]);
      const float y2 = radd(rdot3(a.Rrs[6], a.Rrs[7], a.Rrs[8], x0, x1, x2), a.trs[2]);
      if (y2 > 0.0f) {
        const float uk = radd(rmul(rdiv(y0, y2), a.kfx), a.kcx);
        const float vk = radd(rmul(rdiv(y1, y2), a.kfy), a.kcy);
        if (uk >= 1.0f && vk >= 1.0f && uk < (float)(a.kW - 2) && vk < (float)(a.kH - 2)) {
          const float fu = floorf(uk), fv = floorf(vk);
          const int iu = (int)fu, iv = (int)fv;
          const float au = uk - fu, av = vk - fv;
          const float4 c00 = __ldg(a.kf + iv * a.kW + iu), c10 = __ldg(a.kf + iv * a.kW + iu + 1);
          const float4 c01 = __ldg(a.kf + (iv + 1) * a.kW + iu), c11 = __ldg(a.kf + (iv + 1) * a.kW + iu + 1);
          const float w00 = (1 - au) * (1 - av), w10 = au * (1 - av), w01 = (1 - au) * av, w11 = au * av;
          const float Ik = w00 * c00.x + w10 * c10.x + w01 * c01.x + w11 * c11.x;
          const float gx = w00 * c00.y + w10 * c10.y + w01 * c01.y + w11 * c11.y;
          const float gy = w00 * c00.z + w10 * c10.z + w01 * c01.z + w11 * c11.z;
          const float r = __ldg(a.inten + p) - Ik;
          if (fabsf(r) <= a.thr) {
            // dr/dy = -(gx, gy) d(pi)/dy, then dr/dx = (dr/dy) R_rs
            const float iz = 1.0f / y2;
            const float dy0 = -gx * a.kfx * iz;
            const float dy1 = -gy * a.kfy * iz;
            const float dy2 = (gx * a.kfx * y0 + gy * a.kfy * y1) * iz * iz;
            const float ax0 = dy0 * a.Rrs[0] + dy1 * a.Rrs[3] + dy2 * a.Rrs[6];
            const float ax1 = dy0 * a.Rrs[1] + dy1 * a.Rrs[4] + dy2 * a.Rrs[7];
            const float ax2 = dy0 * a.Rrs[2] + dy1 * a.Rrs[5] + dy2 * a.Rrs[8];
            float J[DIM];
            J[0] = ax0;
            J[1] = ax1;
            J[2] = ax2;
            J[3] = x1 * ax2 - x2 * ax1;
            J[4] = x2 * ax0 - x0 * ax2;
            J[5] = x0 * ax1 - x1 * ax0;
            if (DIM == 7) J[DIM - 1] = ax0 * x0 + ax1 * x1 + ax2 * x2;
            acc.row(J, r, a.lambda * wz);
            acc.v[A::N - 1] += 1.0f;
          }
        }
      }
    }
  }

  // ---- block reduction in a fixed order
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < A::N; ++i) {
    float x = acc.total(i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_red[warp][i] = x;
  }
  __syncthreads();
  if (threadIdx.x < A::N) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < ICP_THREADS / 32; ++w) s += s_red[w][threadIdx.x];
    a.partials[blockIdx.x * A::N + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;

  // ---- last CTA: sum of the partials in a fixed order - PARTS consecutive ranges of CTAs,
  // each summed in CTA order by its own thread, then the range sums in order - then the solve
  // by one warp. A range is summed in double-single arithmetic (FP32 value + FP32 sum of the
  // exact rounding errors of the additions, Knuth's TwoSum: about 48 bits, far below the FP32
  // partials' own error) because GB300's FP64 rate is low; the range sums are added in FP64.
  constexpr int PARTS = ICP_THREADS / A::N;
  __shared__ double s_psum[PARTS][A::N];
  {
    const int G = (int)gridDim.x, chunk = (G + PARTS - 1) / PARTS;
    const int slot = threadIdx.x % A::N, part = threadIdx.x / A::N;
    if (part < PARTS) {
      const int b0 = part * chunk, b1 = min(G, b0 + chunk);
      float hi = 0.0f, lo = 0.0f;
      int b = b0;
      for (; b + 16 <= b1; b += 16) {
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = __ldcg(a.partials + (b + q) * A::N + slot);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const float t = __fadd_rn(hi, v[q]);
          const float bp = __fsub_rn(t, hi);
          const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(v[q], bp));
          hi = t;
          lo = __fadd_rn(lo, e);
        }
      }
      for (; b < b1; ++b) {
        const float x = __ldcg(a.partials + b * A::N + slot);
        const float t = __fadd_rn(hi, x);
        const float bp = __fsub_rn(t, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(x, bp));
        hi = t;
        lo = __fadd_rn(lo, e);
      }
      s_psum[part][slot] = (double)hi + (double)lo;
    }
  }
  __syncthreads();
  if (threadIdx.x < A::N) {
    double s = 0.0;
    for (int q = 0; q < PARTS; ++q) s += s_psum[q][threadIdx.x];
    s_sum[threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  if (threadIdx.x == 0) *a.ticket = 0u;
  const bool stop = icp_solve_update_warp<DIM>(s_sum, DIM, a.pose, a.stats, a.min_rows, a.stop_norm, a.lm);
  if (threadIdx.x == 0 && stop) *a.stop = 1;
}

// ------------------------------------------------------------- batched ----
// Batched registration: one thread-block cluster per problem runs the whole coarse-to-fine
// schedule (levels-1 .. 0, iters[l] Gauss-Newton iterations, early stop per level) in one
// launch. Per iteration the CTAs of the cluster walk the problem's pixels, reduce their rows
// in FP32 (warp shuffles, then warps in a fixed order) into a partial in their shared memory;
// after a cluster barrier, rank 0 adds the partials in FP64 in rank order through distributed
// shared memory, solves and updates the pose; after a second barrier every CTA copies the
// pose and the level decision from rank 0. The published pose is double-buffered by
// iteration parity, so a CTA still copying one iteration's pose cannot see the next one.
// Only hardware cluster barriers are waited on: the CTAs of a cluster are co-scheduled.
namespace cg = cooperative_groups;

constexpr int BATCH_MAX_THREADS = 512;

template <bool KAHAN>
__global__ void __launch_bounds__(BATCH_MAX_THREADS) k_icp_batch(const __grid_constant__ IcpBatchArgs a) {
  using A = Acc<7, KAHAN>;
  cg::cluster_group cl = cg::this_cluster();
  const int CL = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int prob = blockIdx.x / CL;
  __shared__ float s_red[BATCH_MAX_THREADS / 32][A::N];
  __shared__ float s_part[A::N];
  __shared__ double s_sum[A::N];
  __shared__ double s_pose[2][16];  // rank 0: published estimate by iteration parity
  __shared__ int s_done[2];
  __shared__ double s_cur[16];      // this CTA's copy of the estimate
  __shared__ dtsdf_icp_stats s_st;  // rank 0
  if (prob >= a.n) return;  // the whole cluster (no barrier reached)
  const IcpProblemDev& P = a.p[prob];
  const int dsolve = P.sim3 ? 7 : 6;
  const int tid = threadIdx.x, nth = blockDim.x;
  if (tid < 16) s_cur[tid] = P.pose[tid];
  if (rank == 0 && tid == 0) {
    memset(&s_st, 0, sizeof(s_st));
    s_done[0] = s_done[1] = 0;
  }
  __syncthreads();
  int gi = 0;  // iterations run so far (all levels): parity of the published buffers
  for (int l = a.levels - 1; l >= 0; --l) {
    const float* __restrict__ depth = P.depth[l];
    const Intr K = P.K[l];
    const int n = K.W * K.H;
    const float eps2 = rmul(a.eps[l], a.eps[l]);
    for (int it = 0; it < a.iters[l]; ++it, ++gi) {
      float Am[9], tv[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) Am[3 * i + j] = (float)(s_cur[4 * i + j] - (i == j ? 1.0 : 0.0));
        tv[i] = (float)s_cur[4 * i + 3];
      }
      A acc;
      acc.zero();
      for (int p = rank * nth + tid; p < n; p += CL * nth) {
        const float z = __ldg(depth + p);
        if (!(z > 0.0f)) continue;
        float x0, x1, x2, wz;
        geo_row<7, KAHAN>(acc, z, p % K.W, p / K.W, K.fx, K.fy, K.cx, K.cy, Am, tv, P.ref, P.Kr.W, P.Kr.H, P.Kr.fx,
                          P.Kr.fy, P.Kr.cx, P.Kr.cy, eps2, a.zmin, P.sim3 != 0, x0, x1, x2, wz);
      }
      // CTA partial: warp shuffles, then warps in a fixed order
      const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
      for (int i = 0; i < A::N; ++i) {
        float x = acc.total(i);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) s_red[warp][i] = x;
      }
      __syncthreads();
      if (tid < A::N) {
        float sm = 0.f;
        for (int w = 0; w < nth / 32; ++w) sm += s_red[w][tid];
        s_part[tid] = sm;
      }
      cl.sync();  // every partial of the cluster is in place
      const int b = gi & 1;
      if (rank == 0) {
        if (tid < A::N) {
          double sm = 0.0;
          for (int r = 0; r < CL; ++r) sm += (double)*cl.map_shared_rank(&s_part[tid], r);
          s_sum[tid] = sm;
        }
        __syncthreads();
        if (tid < 32) {
          const bool stop = icp_solve_update_warp<7>(s_sum, dsolve, s_cur, &s_st, a.min_rows, a.stop_norm);
          if (tid < 16) s_pose[b][tid] = s_cur[tid];
          if (tid == 0) s_done[b] = stop ? 1 : 0;
        }
      }
      cl.sync();  // the estimate and the level decision are published
      __shared__ int s_stop;
      if (rank != 0 && tid < 16) s_cur[tid] = *cl.map_shared_rank(&s_pose[b][tid], 0);
      if (tid == 0) s_stop = rank == 0 ? s_done[b] : *cl.map_shared_rank(&s_done[b], 0);
      __syncthreads();
      if (s_stop) {
        ++gi;
        break;
      }
    }
  }
  cl.sync();  // rank 0's shared memory stays alive until every copy from it is done
  if (rank == 0 && tid == 0) {
    for (int i = 0; i < 16; ++i) P.pose[i] = s_cur[i];
    if (P.stats) *P.stats = s_st;
  }
}

void launch_icp_batch(const IcpBatchArgs& a, int kahan, int cluster, int threads, cudaStream_t s, cudaError_t* err) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.n * cluster), 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e;
  if (kahan) {
    if (cluster > 8) cudaFuncSetAttribute(k_icp_batch<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    e = cudaLaunchKernelEx(&cfg, k_icp_batch<true>, a);
  } else {
    if (cluster > 8) cudaFuncSetAttribute(k_icp_batch<false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    e = cudaLaunchKernelEx(&cfg, k_icp_batch<false>, a);
  }
  *err = e;
}

// ------------------------------------------------------------ launchers ---
// scale of the intensity sums of level l: 255000 * 4^l
static inline float intensity_scale(int l) { return 255000.0f * (float)(1 << (2 * l)); }

void launch_frame_pyramid(const float4* P, const uint8_t* rgb, int levels, const Intr* K, float* const* depth,
                          float* const* inten, cudaStream_t s) {
  const int n0 = K[0].W * K[0].H;
  k_extract_depth<<<(n0 + 255) / 256, 256, 0, s>>>(P, n0, depth[0]);
  if (rgb) k_intensity<<<(n0 + 255) / 256, 256, 0, s>>>(rgb, n0, inten[0]);
  for (int l = 1; l < levels; ++l) {
    dim3 blk(32, 8), grd((K[l].W + 31) / 32, (K[l].H + 7) / 8);
    k_down<<<grd, blk, 0, s>>>(depth[l - 1], rgb ? inten[l - 1] : nullptr, K[l - 1].W, K[l].W, K[l].H, depth[l],
                               rgb ? inten[l] : nullptr);
  }
  if (rgb)
    for (int l = 0; l < levels; ++l) {
      const int n = K[l].W * K[l].H;
      k_norm_intensity<<<(n + 255) / 256, 256, 0, s>>>(inten[l], n, intensity_scale(l));
    }
}

void launch_keyframe_pyramid(const uint8_t* rgb, int levels, const Intr* K, float* const* tmpI, float4* const* kf,
                             cudaStream_t s) {
  const int n0 = K[0].W * K[0].H;
  k_intensity<<<(n0 + 255) / 256, 256, 0, s>>>(rgb, n0, tmpI[0]);
  for (int l = 1; l < levels; ++l) {
    dim3 blk(32, 8), grd((K[l].W + 31) / 32, (K[l].H + 7) / 8);
    k_down_intensity<<<grd, blk, 0, s>>>(tmpI[l - 1], K[l - 1].W, K[l].W, K[l].H, tmpI[l]);
  }
  for (int l = 0; l < levels; ++l) {
    dim3 blk(32, 8), grd((K[l].W + 31) / 32, (K[l].H + 7) / 8);
    k_kf_grad<<<grd, blk, 0, s>>>(tmpI[l], K[l].W, K[l].H, intensity_scale(l), kf[l]);
  }
}

void launch_icp(const IcpLaunch& L, int sim3, bool photo, int grid, cudaStream_t s) {
  IcpArgs a;
  a.depth = L.depth;
  a.inten = L.inten;
  a.W = L.K.W;
  a.H = L.K.H;
  a.fx = L.K.fx;
  a.fy = L.K.fy;
  a.cx = L.K.cx;
  a.cy = L.K.cy;
  a.ref = L.ref;
  a.rW = L.Kr.W;
  a.rH = L.Kr.H;
  a.rfx = L.Kr.fx;
  a.rfy = L.Kr.fy;
  a.rcx = L.Kr.cx;
  a.rcy = L.Kr.cy;
  a.eps = L.eps;
  a.zmin = L.zmin;
  a.kf = L.kf;
  a.kW = L.Kk.W;
  a.kH = L.Kk.H;
  a.kfx = L.Kk.fx;
  a.kfy = L.Kk.fy;
  a.kcx = L.Kk.cx;
  a.kcy = L.Kk.cy;
  for (int i = 0; i < 9; ++i) a.Rrs[i] = L.Rrs[i];
  for (int i = 0; i < 3; ++i) a.trs[i] = L.trs[i];
  a.Trs_dev = L.Trs_dev;
  a.thr = L.thr;
  a.lambda = L.lambda;
  a.pose = L.pose;
  a.lm = L.lm;
  a.partials = L.partials;
  a.ticket = L.ticket;
  a.stop = L.stop;
  a.stats = L.stats;
  a.min_rows = L.min_rows;
  a.stop_norm = L.stop_norm;
#define DTSDF_ICP(D, P, K) k_icp<D, P, K><<<grid, ICP_THREADS, 0, s>>>(a)
  const bool kahan = L.kahan != 0;
  if (sim3) {
    if (photo) {
      if (kahan) DTSDF_ICP(7, true, true); else DTSDF_ICP(7, true, false);
    } else {
      if (kahan) DTSDF_ICP(7, false, true); else DTSDF_ICP(7, false, false);
    }
  } else {
    if (photo) {
      if (kahan) DTSDF_ICP(6, true, true); else DTSDF_ICP(6, true, false);
    } else {
      if (kahan) DTSDF_ICP(6, false, true); else DTSDF_ICP(6, false, false);
    }
  }
#undef DTSDF_ICP
}

void launch_exp(int dim, const double* xi, double* T, cudaStream_t s) { k_exp<<<1, 32, 0, s>>>(dim, xi, T); }

}  // namespace dtsdf
