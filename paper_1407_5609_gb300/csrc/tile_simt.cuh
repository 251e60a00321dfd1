// FP32 Gram tile mainloop shared by the dense stage and the batched stage: a 128 x 128 tile of
// S = X_I X_J^T (rows row0.. and col0.. of the row-major [rows][Kp] matrix X, Kp % 16 == 0),
// 256 threads, 8 x 8 accumulators per thread, double-buffered shared-memory K slices of 16.
// Thread (tx, ty) owns rows {ty*4 + r, 64 + ty*4 + r} and columns {tx*4 + c, 64 + tx*4 + c}.
#pragma once

namespace cppgb {

constexpr int TILE_BM = 128, TILE_BK = 16, TILE_PAD = 4, TILE_NT = 256;

struct TileSmem {
  float As[2][TILE_BK][TILE_BM + TILE_PAD];
  float Bs[2][TILE_BK][TILE_BM + TILE_PAD];
};

__device__ __forceinline__ void simt_tile_mainloop(const float* __restrict__ X, int64_t Kp, int64_t row0,
                                                   int64_t col0, TileSmem& sm, float (&acc)[8][8]) {
  constexpr int BK = TILE_BK;
  float(&As)[2][TILE_BK][TILE_BM + TILE_PAD] = sm.As;
  float(&Bs)[2][TILE_BK][TILE_BM + TILE_PAD] = sm.Bs;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int lrow = tid >> 2, lk = (tid & 3) * 4;

  const float* Ag = X + (row0 + lrow) * Kp + lk;
  const float* Bg = X + (col0 + lrow) * Kp + lk;
  const int64_t half = 64 * Kp;

#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;

  float4 a0 = *reinterpret_cast<const float4*>(Ag), a1 = *reinterpret_cast<const float4*>(Ag + half);
  float4 b0 = *reinterpret_cast<const float4*>(Bg), b1 = *reinterpret_cast<const float4*>(Bg + half);
  auto stash = [&](int buf) {
    As[buf][lk + 0][lrow] = a0.x; As[buf][lk + 1][lrow] = a0.y; As[buf][lk + 2][lrow] = a0.z; As[buf][lk + 3][lrow] = a0.w;
    As[buf][lk + 0][lrow + 64] = a1.x; As[buf][lk + 1][lrow + 64] = a1.y; As[buf][lk + 2][lrow + 64] = a1.z; As[buf][lk + 3][lrow + 64] = a1.w;
    Bs[buf][lk + 0][lrow] = b0.x; Bs[buf][lk + 1][lrow] = b0.y; Bs[buf][lk + 2][lrow] = b0.z; Bs[buf][lk + 3][lrow] = b0.w;
    Bs[buf][lk + 0][lrow + 64] = b1.x; Bs[buf][lk + 1][lrow + 64] = b1.y; Bs[buf][lk + 2][lrow + 64] = b1.z; Bs[buf][lk + 3][lrow + 64] = b1.w;
  };
  stash(0);
  __syncthreads();

  const int64_t nk = Kp / BK;
  for (int64_t kt = 0; kt < nk; ++kt) {
    const int cur = (int)(kt & 1);
    if (kt + 1 < nk) {
      const int64_t o = (kt + 1) * BK;
      a0 = *reinterpret_cast<const float4*>(Ag + o);
      a1 = *reinterpret_cast<const float4*>(Ag + half + o);
      b0 = *reinterpret_cast<const float4*>(Bg + o);
      b1 = *reinterpret_cast<const float4*>(Bg + half + o);
    }
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float4 ra0 = *reinterpret_cast<const float4*>(&As[cur][k][ty * 4]);
      float4 ra1 = *reinterpret_cast<const float4*>(&As[cur][k][64 + ty * 4]);
      float4 rb0 = *reinterpret_cast<const float4*>(&Bs[cur][k][tx * 4]);
      float4 rb1 = *reinterpret_cast<const float4*>(&Bs[cur][k][64 + tx * 4]);
      float ra[8] = {ra0.x, ra0.y, ra0.z, ra0.w, ra1.x, ra1.y, ra1.z, ra1.w};
      float rb[8] = {rb0.x, rb0.y, rb0.z, rb0.w, rb1.x, rb1.y, rb1.z, rb1.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(ra[r], rb[c], acc[r][c]);
    }
    if (kt + 1 < nk) stash(cur ^ 1);
    __syncthreads();
  }
}

}  // namespace cppgb
