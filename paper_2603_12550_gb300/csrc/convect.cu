// convect.cu -- the convection term of the micro-macro model: transport of a
// field held at the nodes of a structured macroscopic grid by the flow, the
// u . grad_x q term of Eq. model_DymRepPar (and u . grad_x p of Eq.
// model_DymReduced for reduced coordinates), which the homogeneous-flow
// experiments of Sec. 3 drop and a grid of ensembles needs (include/
// vds_batch.h, vds_convect).
//
// One first-order upwind step per call:
//   Q_out[g] = Q[g] - dt sum_b ( max(u_b,0) (Q[g] - Q[g - e_b])
//                               + min(u_b,0) (Q[g + e_b] - Q[g]) ) / dx_b
// in FP32 (the field is FP32; each output is a handful of operations on
// values of the same magnitude).  The field is M values per node, node-major,
// so the CTA of (node g, a range of values) reads the same range of each
// neighbour node: every access is coalesced.  The node is the fastest grid
// index, so the CTAs resident at one time cover one or two value ranges of
// every node (4 KB each): the neighbours' copies of a range are read from L2
// while it is still there, whatever the field's size, and HBM sees one read
// and one write of the field, its bound.
#include "vds_internal.cuh"

#include "vds_batch.h"

namespace {

constexpr int CV_NT = 256;
constexpr int CV_PER = 8;  // values per thread

__global__ void __launch_bounds__(CV_NT)
    k_convect(const float *__restrict__ q, float *__restrict__ out, int nx, int ny, int nz, long M,
              const float *__restrict__ u, float cx, float cy, float cz, int bc) {
  const int g = blockIdx.x;
  const int G = nx * ny * nz;
  if (g >= G) return;
  const int ix = g % nx, iy = (g / nx) % ny, iz = g / (nx * ny);
  // neighbour nodes below and above along each axis (periodic or clamped)
  auto nb = [&](int i, int n, int d) -> int {
    int j = i + d;
    if (j < 0) j = bc == 0 ? n - 1 : 0;
    if (j >= n) j = bc == 0 ? 0 : n - 1;
    return j;
  };
  const int gxm = nb(ix, nx, -1) + nx * (iy + ny * iz), gxp = nb(ix, nx, 1) + nx * (iy + ny * iz);
  const int gym = ix + nx * (nb(iy, ny, -1) + ny * iz), gyp = ix + nx * (nb(iy, ny, 1) + ny * iz);
  const int gzm = ix + nx * (iy + ny * nb(iz, nz, -1)), gzp = ix + nx * (iy + ny * nb(iz, nz, 1));
  // Courant factors dt u_b / dx_b; the upwind neighbour of each axis (the
  // sign of u_b is the same for the whole CTA, so each value reads the node
  // itself and at most three neighbours)
  const float ux = nx > 1 ? u[(size_t)g * 3] * cx : 0.f;
  const float uy = ny > 1 ? u[(size_t)g * 3 + 1] * cy : 0.f;
  const float uz = nz > 1 ? u[(size_t)g * 3 + 2] * cz : 0.f;
  const float *qx = ux > 0.f ? q + (size_t)gxm * M : ux < 0.f ? q + (size_t)gxp * M : nullptr;
  const float *qy = uy > 0.f ? q + (size_t)gym * M : uy < 0.f ? q + (size_t)gyp * M : nullptr;
  const float *qz = uz > 0.f ? q + (size_t)gzm * M : uz < 0.f ? q + (size_t)gzp * M : nullptr;
  const float *qg = q + (size_t)g * M;
  const long chunk = (long)blockIdx.y + (long)gridDim.y * blockIdx.z;
  const long m0 = chunk * CV_NT * CV_PER + threadIdx.x;
  if (m0 >= M) return;
  float *og = out + (size_t)g * M;
  // u_b > 0: u_b (Q[g] - Q[g - e_b]); u_b < 0: u_b (Q[g + e_b] - Q[g])
  auto upd = [](float d, float ub, float c, float v) { return d + (ub > 0.f ? ub * (c - v) : ub * (v - c)); };
  if (m0 + (long)(CV_PER - 1) * CV_NT < M) {
    // a full chunk: every load is issued before the arithmetic (memory-level
    // parallelism is what bounds this kernel)
    float c[CV_PER], vx[CV_PER], vy[CV_PER], vz[CV_PER];
#pragma unroll
    for (int k = 0; k < CV_PER; ++k) {
      const long m = m0 + (long)k * CV_NT;
      c[k] = qg[m];
      vx[k] = qx ? qx[m] : 0.f;
      vy[k] = qy ? qy[m] : 0.f;
      vz[k] = qz ? qz[m] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < CV_PER; ++k) {
      float d = 0.f;
      if (qx) d = upd(d, ux, c[k], vx[k]);
      if (qy) d = upd(d, uy, c[k], vy[k]);
      if (qz) d = upd(d, uz, c[k], vz[k]);
      og[m0 + (long)k * CV_NT] = c[k] - d;
    }
    return;
  }
  for (int k = 0; k < CV_PER; ++k) {
    const long m = m0 + (long)k * CV_NT;
    if (m >= M) break;
    const float ck = qg[m];
    float d = 0.f;
    if (qx) d = upd(d, ux, ck, qx[m]);
    if (qy) d = upd(d, uy, ck, qy[m]);
    if (qz) d = upd(d, uz, ck, qz[m]);
    og[m] = ck - d;
  }
}

}  // namespace

extern "C" int vds_convect(vds_ctx *c, const float *q_in, float *q_out, int nx, int ny, int nz, long M,
                           const float *u, const double *dx, double dt, int bc) {
  if (!c || !q_in || !q_out || !u || !dx || nx < 1 || ny < 1 || nz < 1 || M < 1) return VDS_EARG;
  if (!(dt > 0.0) || (bc != 0 && bc != 1)) return VDS_EARG;
  for (int b = 0; b < 3; ++b)
    if (!(dx[b] > 0.0)) return VDS_EARG;
  const long long G = (long long)nx * ny * nz;
  if (G > (1ll << 30)) return VDS_EARG;
  const size_t bytes = (size_t)G * (size_t)M * sizeof(float);
  const char *a0 = (const char *)q_in, *b0 = (const char *)q_out;
  if (a0 < b0 + bytes && b0 < a0 + bytes) return VDS_EARG;  // in place is not supported
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return VDS_ECUDA;
  if (prev != c->device && cudaSetDevice(c->device) != cudaSuccess) return VDS_ECUDA;
  const long chunks = (M + CV_NT * CV_PER - 1) / (CV_NT * CV_PER);
  const unsigned gy = (unsigned)(chunks < 65535 ? chunks : 65535);
  const long gz = (chunks + gy - 1) / gy;
  int st = VDS_OK;
  if (gz > 65535) {
    st = VDS_EARG;
  } else {
    k_convect<<<dim3((unsigned)G, gy, (unsigned)gz), CV_NT, 0, c->stream>>>(
        q_in, q_out, nx, ny, nz, M, u, (float)(dt / dx[0]), (float)(dt / dx[1]), (float)(dt / dx[2]), bc);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      vds_last_cuda_error(e);
      st = VDS_ECUDA;
    } else {
      ++c->launches;
    }
  }
  if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
  return st;
}
