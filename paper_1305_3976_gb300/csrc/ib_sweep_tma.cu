// Strided line solves (y and z lines, Steps 3c-3e and the Sec. 6.1 solves)
// for FP32 fields with the lines staged in shared memory by the Tensor Memory
// Accelerator.
//
// A slab is 32 adjacent x columns of one field times whole lines along the
// solve axis at one value of the remaining coordinate.  One thread copies a
// slab in with 3D bulk tensor copies (one box, or two when a line is longer
// than the 256-element box limit) that complete on an mbarrier, and copies
// the solved slab out with bulk tensor stores.  The solve is the one of
// k_sweep_s with one column per lane: warp w holds elements w CH .. w CH +
// CH - 1 of its lane's line in registers, runs the local recurrences of both
// factors of (I - lam S)(I - lam S^-1) and the chunk scans through shared
// memory, then the periodic corrections (the factorization of Sec. 4.2's
// cyclic system into two bidiagonal factors).
//
// Persistent CTAs (one per SM for 512-long lines) loop over the slabs with
// three stages: the copy-in of the next slab, the arithmetic on the current
// one and the copy-out of the previous one overlap.  Waits on the mbarriers
// are bounded: on timeout the CTA sets a process-wide flag (reported by
// ib_diagnostics as IB_ERR_TIMEOUT), waits once more for its copies and
// returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "ib_internal.cuh"

namespace ibg {

namespace {

constexpr int kStages = 3;
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s

__device__ int g_wait_timeout = 0;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t *b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void bar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bar_expect(uint64_t *b, uint32_t bytes) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(su32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t *b, uint32_t parity) {
  uint32_t done;
  asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(done)
               : "r"(su32(b)), "r"(parity)
               : "memory");
  return done != 0;
}
__device__ __forceinline__ unsigned long long gtime_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// wait for the phase with the given parity, at most limit_ns nanoseconds
__device__ __forceinline__ bool bar_wait(uint64_t *b, uint32_t parity, unsigned long long limit_ns = kWaitNs) {
  const unsigned long long t0 = gtime_ns();
  while (!bar_try(b, parity))
    if (gtime_ns() - t0 > limit_ns) return false;
  return true;
}
__device__ __forceinline__ void tma_in(float *dst, const CUtensorMap *m, int x, int y, int z, uint64_t *b) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(su32(b))
      : "memory");
}
__device__ __forceinline__ void tma_out(const CUtensorMap *m, int x, int y, int z, const float *src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<uint64_t>(m)),
               "r"(x), "r"(y), "r"(z), "r"(su32(src))
               : "memory");
}
__device__ __forceinline__ void tma_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// at most N committed copy-outs may still be reading shared memory
template <int N>
__device__ __forceinline__ void tma_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void tma_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

}  // namespace

template <int CH, int W, bool FULL, bool EXT>
__global__ void __launch_bounds__(32 * W, 1) k_sweep_tma(const __grid_constant__ SweepTmaMaps maps,
                                                         const SweepArgs<float> a, const int axis, const int nbox,
                                                         const int boxlen) {
  pdl_wait();
  pdl_release();
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ float sz[W][33];
  __shared__ float lp[CH + 1];  // lam^0 .. lam^CH
  __shared__ int s_ok;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nx = a.n[0], nl = a.n[axis];
  const int slabf = 32 * nbox * boxlen;  // floats per slab (a multiple of 32)
  float *const stage0 = reinterpret_cast<float *>(sm);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + (size_t)kStages * slabf * sizeof(float));
  const int nxb = (nx + 31) / 32;
  const int nother = axis == 1 ? (a.dim == 3 ? a.n[2] : 1) : a.n[1];
  const int per_field = nxb * nother;
  const int nslab = per_field * maps.nfields;
  const uint32_t bytes = (uint32_t)slabf * (uint32_t)sizeof(float);
  auto coords = [&](int slab, int b, int &x, int &y, int &z, int &f) {
    f = slab / per_field;
    const int r = slab - f * per_field;
    const int xb = r % nxb, other = r / nxb;
    x = 32 * xb;
    if (axis == 1) {
      y = b * boxlen;
      z = other;
    } else {
      y = other;
      z = b * boxlen;
    }
  };
  auto load = [&](int slab, int st) {  // thread 0
    tma_wait_read<1>();  // the copy-out two slabs back has read this stage
    proxy_fence();
    bar_expect(bar + st, bytes);
    for (int b = 0; b < nbox; ++b) {
      int x, y, z, f;
      coords(slab, b, x, y, z, f);
      tma_in(stage0 + st * slabf + b * 32 * boxlen, &maps.in[f], x, y, z, bar + st);
    }
  };
  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) bar_init(bar + st);
    bar_init_fence();
    if ((int)blockIdx.x < nslab) load(blockIdx.x, 0);
  }
  if (threadIdx.x <= CH) lp[threadIdx.x] = a.co.pw[threadIdx.x];
  __syncthreads();
  const float lam = a.co.lam, gCH = lp[CH];
  const float *pw = a.co.pw;
  const int start = w * CH;
  const int len = FULL ? CH : max(0, min(CH, nl - start));
  uint32_t parity = 0u;  // bit st: phase of stage st's barrier
  int st = 0;
  for (int slab = blockIdx.x; slab < nslab; slab += gridDim.x, st = st + 1 == kStages ? 0 : st + 1) {
    if (threadIdx.x == 0) {
      const int nxt = slab + gridDim.x;
      if (nxt < nslab) load(nxt, st + 1 == kStages ? 0 : st + 1);
      const bool ok = bar_wait(bar + st, (parity >> st) & 1u);
      if (!ok) {
        atomicExch(&g_wait_timeout, 1);
        for (int q = 0; q < kStages; ++q) bar_wait(bar + q, (parity >> q) & 1u);
        tma_wait_all();
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;
    parity ^= 1u << st;
    float *sl = stage0 + st * slabf;
    float v[CH];
#pragma unroll
    for (int e = 0; e < CH; ++e) v[e] = (FULL || e < len) ? sl[(start + e) * 32 + lane] : 0.f;
    // forward factor (I - lam S) y = b: local pass, chunk scan, correction
    {
      float z = 0.f;
#pragma unroll
      for (int e = 0; e < CH; ++e)
        if (FULL || e < len) v[e] = z = fmaf(lam, z, v[e]);
      sz[w][lane] = z;
    }
    __syncthreads();
    {
      const float pstart = pw[min(start, nl)];
      float cin = 0.f;
      for (int q = 0; q < w; ++q) cin = fmaf(cin, FULL ? gCH : pw[max(0, min(CH, nl - q * CH))], sz[q][lane]);
      float tot = cin;
      for (int q = w; q < W; ++q) tot = fmaf(tot, FULL ? gCH : pw[max(0, min(CH, nl - q * CH))], sz[q][lane]);
      const float t = EXT ? wrap_term<true>(a.co, min(start, nl), tot, cin) : fmaf(pstart, tot * a.co.inv_1m, cin);
#pragma unroll
      for (int e = 0; e < CH; ++e)
        if (FULL || e < len) v[e] = fmaf(lp[e + 1], t, v[e]);
    }
    __syncthreads();
    // backward factor (I - lam S^-1) x = y
    {
      float z = 0.f;
#pragma unroll
      for (int e = CH - 1; e >= 0; --e)
        if (FULL || e < len) v[e] = z = fmaf(lam, z, v[e]);
      sz[w][lane] = z;
    }
    __syncthreads();
    if (FULL || len > 0) {
      const float pend = pw[nl - start - len];
      float cin = 0.f;
      for (int q = W - 1; q > w; --q) cin = fmaf(cin, FULL ? gCH : pw[max(0, min(CH, nl - q * CH))], sz[q][lane]);
      float tot = cin;
      for (int q = w; q >= 0; --q) tot = fmaf(tot, FULL ? gCH : pw[max(0, min(CH, nl - q * CH))], sz[q][lane]);
      const float t = EXT ? wrap_term<true>(a.co, nl - start - len, tot, cin) : fmaf(pend, tot * a.co.inv_1m, cin);
#pragma unroll
      for (int e = 0; e < CH; ++e)
        if (FULL || e < len) {
          const int pe = FULL ? CH - e : max(0, len - e);
          sl[(start + e) * 32 + lane] = fmaf(lp[pe], t, v[e]) * a.co.scale;
        }
    }
    proxy_fence();  // this thread's results before the copy-out reads them
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int b = 0; b < nbox; ++b) {
        int x, y, z, f;
        coords(slab, b, x, y, z, f);
        tma_out(&maps.out[f], x, y, z, sl + b * 32 * boxlen);
      }
      tma_commit();
    }
  }
  if (threadIdx.x == 0) tma_wait_all();
}

namespace {

typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                             const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, looked up once per process (thread-safe)
EncodeFn encoder() {
  static std::once_flag once;
  static EncodeFn fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeFn)p;
  });
  return fn;
}

// box length along the solve axis: the whole line, or half of it for lines
// longer than the 256-element box limit
int box_len(int nl) { return nl <= 256 ? nl : nl / 2; }

bool encode(CUtensorMap *m, const float *base, const SweepArgs<float> &a, int axis, int boxlen) {
  EncodeFn enc = encoder();
  if (!enc) return false;
  const int nz = a.dim == 3 ? a.n[2] : 1;
  const cuuint64_t dim[3] = {(cuuint64_t)a.n[0], (cuuint64_t)a.n[1], (cuuint64_t)nz};
  const cuuint64_t stride[2] = {(cuuint64_t)a.n[0] * sizeof(float), (cuuint64_t)a.n[0] * a.n[1] * sizeof(float)};
  const cuuint32_t box[3] = {32u, axis == 1 ? (cuuint32_t)boxlen : 1u, axis == 2 ? (cuuint32_t)boxlen : 1u};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)base, dim, stride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct TmaShape {
  int ch, w;
};
TmaShape tma_shape(int nl) {
  if (nl <= 64) return {8, 8};
  if (nl <= 128) return {16, 8};
  if (nl <= 256) return {16, 16};
  return {16, 32};
}

}  // namespace

// The TMA sweep applies to FP32 y and z lines with rows of a multiple of 4
// floats (16-byte row strides) and lines of at most 256 elements or of even
// length (two boxes).
bool sweep_tma_ok(const SweepArgs<float> &a, int axis) {
  if (axis == 0 || a.n[0] % 4 != 0) return false;
  const int nl = a.n[axis];
  return nl <= 256 || nl % 2 == 0;
}

void sweep_tma_shape(int nl, int *ch, int *w) {
  const TmaShape t = tma_shape(nl);
  *ch = t.ch;
  *w = t.w;
}

// One CTA arms an mbarrier for 16 bytes that no copy will deliver and waits
// for it with a limit of limit_ns: the wait runs out and sets the flag.
__global__ void k_wait_selftest(unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  bar_init(&bar);
  bar_init_fence();
  bar_expect(&bar, 16);
  if (!bar_wait(&bar, 0, limit_ns)) atomicExch(&g_wait_timeout, 1);
}

cudaError_t launch_wait_selftest(unsigned long long limit_ns, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(limit_ns);
  return cudaGetLastError();
}

int take_wait_timeout() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_wait_timeout, sizeof(int)) != cudaSuccess) return 0;
  if (v) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_wait_timeout, &zero, sizeof(int));
  }
  return v;
}

cudaError_t launch_sweep_tma(int axis, int nfields, const SweepArgs<float> &a, cudaStream_t s) {
  const int nl = a.n[axis], boxlen = box_len(nl), nbox = (nl + boxlen - 1) / boxlen;
  SweepTmaMaps maps;
  maps.nfields = nfields;
  for (int f = 0; f < nfields; ++f) {
    const float *in = a.fin[f] ? a.fin[f] : a.f[f];
    if (!encode(&maps.in[f], in, a, axis, boxlen) || !encode(&maps.out[f], a.f[f], a, axis, boxlen))
      return cudaErrorInvalidValue;
  }
  const size_t smem = (size_t)kStages * 32 * nbox * boxlen * sizeof(float) + kStages * sizeof(uint64_t);
  // SM count of the current device, queried on every call (devices may differ)
  int sms = 0, dev = 0;
  {
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  const int nother = axis == 1 ? (a.dim == 3 ? a.n[2] : 1) : a.n[1];
  const int nslab = (a.n[0] + 31) / 32 * nother * nfields;
  auto run = [&](auto kernel, int threads) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int ctas = nslab < sms * per_sm ? nslab : sms * per_sm;
    return launch_pdl(kernel, dim3(ctas), dim3(threads), smem, s, maps, a, axis, nbox, boxlen);
  };
  const TmaShape t = tma_shape(nl);
  const bool full = t.ch * t.w == nl;
#define IBG_TMA(CH, W)                                                                                     \
  if (t.ch == CH && t.w == W) {                                                                      \
    if (a.co.wrap_ext)                                                                               \
      return full ? run(k_sweep_tma<CH, W, true, true>, 32 * W) : run(k_sweep_tma<CH, W, false, true>, 32 * W); \
    return full ? run(k_sweep_tma<CH, W, true, false>, 32 * W) : run(k_sweep_tma<CH, W, false, false>, 32 * W); \
  }
  IBG_TMA(8, 8)
  IBG_TMA(16, 8)
  IBG_TMA(16, 16)
  IBG_TMA(16, 32)
#undef IBG_TMA
  return cudaErrorInvalidValue;
}

}  // namespace ibg
