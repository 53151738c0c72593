// The directional (normal-weighted) confocal model of Sec. 2 for a given
// normal field n = (a, b, c): tau(x', t) = sum over x of u(x) ((x' - x) . n(x)
// / d)^2 / d^4 delta(2 d - t c), the confocal case of the paper's
// non-confocal direction-albedo model (illumination and detection at the
// same wall point).  With lateral coordinates X, Y and depth Z in units of
// the range R, g = X a + Y b + Z c and (x' - x) . n = X' a + Y' b - g, the
// squared cosine expands into six products of a field on the voxel grid and
// a weight on the scan point:
//     X'^2 a^2 + Y'^2 b^2 + g^2 + 2 X'Y' a b - 2 X' a g - 2 Y' b g,
// and on the support of the delta d / R = rho_t = (k + 1/2) / nt for time
// bin k.  So the operator is sum_t w_t(x', k) A(f_t u) with the albedo
// operator A of Eq. 3 (R_t^{-1} H R_z, the plan's kernels unchanged), and
// its transpose sum_t f_t A^T(w_t tau).  Two field-sized scratch buffers of
// the plan (allocated on first use) hold one term at a time.
#include <algorithm>

#include "passes.cuh"

namespace nlos {

namespace {

constexpr int kDirTerms = 6;

struct DirGeom {
  int nx, ny, nt;
  float sx, sy;   // lateral spacing in units of R
  float inv_nt;
};

__device__ __forceinline__ float lat(int i, int n, float s) { return ((float)i + 0.5f - 0.5f * (float)n) * s; }

// Field factor f_t(x) of term t at voxel (i, j, k) with normal (a, b, c).
__device__ __forceinline__ float dir_field(int t, float X, float Y, float Z, float a, float b, float c) {
  const float g = X * a + Y * b + Z * c;
  switch (t) {
    case 0: return a * a;
    case 1: return b * b;
    case 2: return g * g;
    case 3: return a * b;
    case 4: return a * g;
    default: return b * g;
  }
}
// Weight w_t(x', k) of term t at scan point (i, j), time bin k.
__device__ __forceinline__ float dir_weight(int t, float X, float Y, float rho) {
  const float inv = 1.0f / (rho * rho);
  switch (t) {
    case 0: return X * X * inv;
    case 1: return Y * Y * inv;
    case 2: return inv;
    case 3: return 2.0f * X * Y * inv;
    case 4: return -2.0f * X * inv;
    default: return -2.0f * Y * inv;
  }
}

// out = f_t u (forward input), or acc += f_t v (adjoint output).
__global__ void k_dir_field(const float* __restrict__ v, const float* __restrict__ normals, DirGeom G, int t,
                            float* __restrict__ out, int accumulate) {
  const size_t V = (size_t)G.nx * G.ny * G.nt;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < V; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % G.nt);
    const size_t col = e / G.nt;
    const int j = (int)(col % G.ny), i = (int)(col / G.ny);
    const float f = dir_field(t, lat(i, G.nx, G.sx), lat(j, G.ny, G.sy), ((float)k + 0.5f) * G.inv_nt, normals[e],
                              normals[V + e], normals[2 * V + e]);
    out[e] = accumulate ? out[e] + f * v[e] : f * v[e];
  }
}

// Forward: tau (+)= w_t y on every column (zero on unsampled columns when
// colpos is given).  Adjoint: out = w_t r (r zeroed on unsampled columns).
__global__ void k_dir_weight(const float* __restrict__ y, DirGeom G, int t, const int32_t* __restrict__ colpos,
                             float* __restrict__ out, int accumulate) {
  const size_t V = (size_t)G.nx * G.ny * G.nt;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < V; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % G.nt);
    const size_t col = e / G.nt;
    const int j = (int)(col % G.ny), i = (int)(col / G.ny);
    const bool live = colpos == nullptr || __ldg(colpos + col) >= 0;
    const float w = live ? dir_weight(t, lat(i, G.nx, G.sx), lat(j, G.ny, G.sy), ((float)k + 0.5f) * G.inv_nt) : 0.f;
    out[e] = accumulate ? out[e] + w * y[e] : w * y[e];
  }
}

DirGeom dir_geom(const Plan& P) {
  DirGeom G;
  G.nx = P.nx;
  G.ny = P.ny;
  G.nt = P.nt;
  G.sx = (float)(P.wall_width_m / P.nx / P.range_m);
  G.sy = (float)(P.wall_width_m / P.ny / P.range_m);
  G.inv_nt = 1.0f / (float)P.nt;
  return G;
}

nlos_status dir_scratch(Plan& P) {
  const size_t F = (size_t)P.nx * P.ny * P.nt * sizeof(float);
  for (int i = 0; i < 2; ++i)
    if (!P.d_dir[i] && cudaMalloc(&P.d_dir[i], F) != cudaSuccess) {
      cudaGetLastError();
      P.d_dir[i] = nullptr;
      return fail(NLOS_ERR_OOM, "directional model: scratch buffers");
    }
  return NLOS_OK;
}

int dir_grid(size_t n) { return (int)std::min<size_t>((n + 255) / 256, (size_t)device_sm_count() * 16); }

}  // namespace

nlos_status apply_forward_directional(Plan& P, const float* u, const float* normals, float* tau, bool masked,
                                      cudaStream_t st) {
  NLOS_TRY(dir_scratch(P));
  const DirGeom G = dir_geom(P);
  const size_t V = (size_t)P.nx * P.ny * P.nt;
  const int32_t* colpos = masked && !P.full_mask ? P.d_colpos : nullptr;
  for (int t = 0; t < kDirTerms; ++t) {
    k_dir_field<<<dir_grid(V), 256, 0, st>>>(u, normals, G, t, P.d_dir[0], 0);
    NLOS_LAUNCH_CHECK("k_dir_field");
    NLOS_TRY(apply_forward(P, P.d_dir[0], P.d_dir[1], false, st));
    k_dir_weight<<<dir_grid(V), 256, 0, st>>>(P.d_dir[1], G, t, colpos, tau, t > 0 ? 1 : 0);
    NLOS_LAUNCH_CHECK("k_dir_weight");
  }
  return NLOS_OK;
}

nlos_status apply_adjoint_directional(Plan& P, const float* tau, const float* normals, float* u, bool masked,
                                      cudaStream_t st) {
  NLOS_TRY(dir_scratch(P));
  const DirGeom G = dir_geom(P);
  const size_t V = (size_t)P.nx * P.ny * P.nt;
  const int32_t* colpos = masked && !P.full_mask ? P.d_colpos : nullptr;
  for (int t = 0; t < kDirTerms; ++t) {
    k_dir_weight<<<dir_grid(V), 256, 0, st>>>(tau, G, t, colpos, P.d_dir[0], 0);
    NLOS_LAUNCH_CHECK("k_dir_weight");
    NLOS_TRY(apply_adjoint(P, P.d_dir[0], P.d_dir[1], false, st));
    k_dir_field<<<dir_grid(V), 256, 0, st>>>(P.d_dir[1], normals, G, t, u, t > 0 ? 1 : 0);
    NLOS_LAUNCH_CHECK("k_dir_field");
  }
  return NLOS_OK;
}

}  // namespace nlos
