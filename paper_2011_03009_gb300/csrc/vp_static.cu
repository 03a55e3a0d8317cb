// Allocation-free volume potential for small grids: vp_apply_static.
//
// Some callers cannot call cudaMalloc: code running while a CUDA stream is being
// captured into a graph (cudaMalloc and cudaFree are not capturable and cudaFree
// synchronises the device), host applications whose device memory is owned by
// another allocator that already holds it all, and latency-bound loops that cannot
// afford the device-wide synchronisation of cudaMalloc/cudaFree.  This entry point
// evaluates u = V_k[f] like vp_plan + vp_kernel_fft + vp_apply, but keeps every
// intermediate (tables, kernel lattice, spectrum octant, FFT workspace) in one
// file-scope __device__ array of fixed size, so it never allocates device memory.
//
// Limits and sharing: grids up to kStaticMaxN voxels per axis (embedding M <= 128).
// Every GPU that loads libvp.so holds the array (about 18.2 MiB) until the process
// exits.  All calls on a device share the array and every call rewrites all of it
// that it reads, so nothing carries over from one call to the next; two calls whose
// GPU work overlaps (different streams, or different host threads) race on it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "vp.h"
#include "vp_internal.cuh"

namespace {

constexpr int kStaticMaxN = VP_STATIC_MAX_N;
constexpr int kStaticMaxM = 2 * kStaticMaxN;  // 128 = 2^7 is 5-smooth
constexpr int kStaticMaxO = kStaticMaxM / 2 + 1;
constexpr double kPi = 3.141592653589793238462643383279502884;

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
// region offsets in bytes
constexpr size_t kOffCube = 0;  // lattice cube M^3, later FFT workspace A and B
constexpr size_t kCubeBytes = (size_t)kStaticMaxM * kStaticMaxM * kStaticMaxM * sizeof(float2);
constexpr size_t kOffOct = align256(kOffCube + kCubeBytes);
constexpr size_t kOctBytes = (size_t)kStaticMaxO * kStaticMaxO * kStaticMaxO * sizeof(float2);
constexpr size_t kOffTw = align256(kOffOct + kOctBytes);
constexpr size_t kTwBytes = 3 * (size_t)kStaticMaxM * sizeof(float2);
constexpr size_t kOffPos = align256(kOffTw + kTwBytes);
constexpr size_t kPosBytes = 3 * (size_t)kStaticMaxM * sizeof(int);
constexpr size_t kOffFold = align256(kOffPos + kPosBytes);
constexpr size_t kFoldBytes = 3 * (size_t)kStaticMaxM * sizeof(int);
constexpr size_t kMaxTiles = ((size_t)kStaticMaxO * kStaticMaxO + 3) / 4;
constexpr size_t kOffTiles = align256(kOffFold + kFoldBytes);
constexpr size_t kTilesBytes = kMaxTiles * 20 * sizeof(int);
constexpr size_t kScratchBytes = align256(kOffTiles + kTilesBytes);

static_assert(kCubeBytes >= ((size_t)kStaticMaxM * kStaticMaxN * kStaticMaxN +
                             (size_t)kStaticMaxM * kStaticMaxM * kStaticMaxN) * sizeof(float2),
              "FFT workspace must fit in the lattice cube region");

// The scratch.  Host code must not take its address directly (that would be the
// host-side shadow, not device memory): it goes through cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

// The array's device address belongs to the CUDA context that loaded the module: after
// cudaDeviceReset, or once the primary context is released and created again, the
// module is loaded anew and the array may sit elsewhere.  The address is therefore
// cached per device together with the context it was taken in, and looked up again
// whenever the current context differs.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return (CtxGetCurrentFn)f;
  }();
  return fn;
}

// The context current on this thread, or nullptr if none is (or it cannot be read).
CUcontext current_context() {
  CtxGetCurrentFn get = ctx_get_current();
  CUcontext c = nullptr;
  if (!get || get(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

struct ScratchAddr {
  CUcontext ctx;
  void* ptr;
};
std::mutex g_addr_mu;
ScratchAddr g_addr[64] = {};

// Device address of the scratch for the current device and context.  The lookup runs
// on the first call in each context; later calls in that context read the cache.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VP_ERR_CUDA;
  if (dev < 0 || dev >= 64) return VP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_addr_mu);
  CUcontext ctx = current_context();
  if (!ctx || g_addr[dev].ctx != ctx || !g_addr[dev].ptr) {
    void* ptr = nullptr;
    // cudaGetSymbolAddress makes the device's primary context current if none is
    if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) return VP_ERR_CUDA;
    ctx = current_context();
    g_addr[dev] = ScratchAddr{ctx, ctx ? ptr : nullptr};  // without a context handle: no caching
    *out = ptr;
    return VP_OK;
  }
  *out = g_addr[dev].ptr;
  return VP_OK;
}

bool smooth5(int v) {
  for (int p : {2, 3, 5})
    while (v % p == 0) v /= p;
  return v == 1;
}

int default_m(int n) {
  int m = 2 * n;
  while (!smooth5(m)) m += 2;
  return m;
}

int default_schedule(int L, int* out) {
  int a = 0, b = 0, c = 0, v = L;
  while (v % 2 == 0) { v /= 2; ++a; }
  while (v % 3 == 0) { v /= 3; ++b; }
  while (v % 5 == 0) { v /= 5; ++c; }
  if (v != 1) return 0;
  int np = 0;
  const int p2 = (a + 3) / 4;
  for (int i = 0; i < p2; ++i) out[np++] = 1 << (a / p2 + (i < a % p2 ? 1 : 0));
  for (int i = 0; i < c; ++i) out[np++] = 5;
  for (int i = 0; i < b; ++i) out[np++] = 3;
  for (int i = np; i < vp::kMaxPass; ++i) out[i] = 0;
  return np;
}

struct StaticTables {
  float2* tw[3];
  int* pos[3];
  int* fold[3];
  int* tiles;
  int m[3];
  int npass[3];
  int radix[3][vp::kMaxPass];
  int ox, oy, ntiles;
};

// Position of frequency f after the DIF passes: digits of f in radices R0, R1, ...
// (least significant first) weighted by the strides s_i = M / (R0 ... Ri).
__device__ int dif_position(const StaticTables& t, int a, int f) {
  int pos = 0, stride = t.m[a];
  for (int i = 0; i < t.npass[a]; ++i) {
    const int R = t.radix[a][i];
    stride /= R;
    pos += (f % R) * stride;
    f /= R;
  }
  return pos;
}

// Frequency held at position pp after the DIF passes (inverse of dif_position).
__device__ int dif_frequency(const StaticTables& t, int a, int pp) {
  int f = 0, mul = 1, stride = t.m[a];
  for (int i = 0; i < t.npass[a]; ++i) {
    const int R = t.radix[a][i];
    stride /= R;
    f += ((pp / stride) % R) * mul;
    mul *= R;
  }
  return f;
}

// Fill every table the sweeps read: twiddles, frequency/position maps and the z tiles.
__global__ void static_tables_kernel(StaticTables t) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthreads = gridDim.x * blockDim.x;
  for (int a = 0; a < 3; ++a) {
    const int M = t.m[a];
    for (int i = tid; i < M; i += nthreads) {
      double s, c;
      sincospi(2.0 * (double)i / (double)M, &s, &c);
      t.tw[a][i] = make_float2((float)c, (float)-s);
      t.pos[a][i] = dif_position(t, a, i);
      const int f = dif_frequency(t, a, i);
      t.fold[a][i] = min(f, M - f);
    }
  }
  const int groups = t.ox * t.oy;
  for (int g = tid; g < 4 * t.ntiles; g += nthreads) {
    int* slot = t.tiles + (size_t)(g / 4) * 20 + (g % 4) * 4;
    int* oct = t.tiles + (size_t)(g / 4) * 20 + 16 + (g % 4);
    int k = 0;
    if (g < groups) {
      const int ox = g / t.oy, oy = g % t.oy;
      const int fx[2] = {ox, t.m[0] - ox};
      const int fy[2] = {oy, t.m[1] - oy};
      const int nfx = (ox == 0 || 2 * ox == t.m[0]) ? 1 : 2;
      const int nfy = (oy == 0 || 2 * oy == t.m[1]) ? 1 : 2;
      for (int i = 0; i < nfx; ++i)
        for (int j = 0; j < nfy; ++j)
          slot[k++] = dif_position(t, 0, fx[i] % t.m[0]) * t.m[1] + dif_position(t, 1, fy[j] % t.m[1]);
      *oct = ox * t.oy + oy;
    } else {
      *oct = -1;
    }
    for (; k < 4; ++k) slot[k] = -1;
  }
}

}  // namespace

extern "C" VP_API int vp_apply_static(const vp_grid* g, int harmonic_n, double f0_hz, const vp_medium* med,
                                      const void* f, void* u, vp_stream_t stream) {
  if (!g || !med || !f || !u || harmonic_n < 1 || !(f0_hz > 0) || !std::isfinite(f0_hz) ||
      !(g->h > 0) || !std::isfinite(g->h) || !(med->c0 > 0) || !(med->rho0 > 0) || !(med->alpha0 >= 0) ||
      !std::isfinite(med->c0) || !std::isfinite(med->rho0) || !std::isfinite(med->alpha0) ||
      !std::isfinite(med->beta) || !std::isfinite(med->eta))
    return VP_ERR_ARG;
  for (int a = 0; a < 3; ++a) {
    if (g->n[a] < 1) return VP_ERR_ARG;
    if (g->n[a] > kStaticMaxN) return VP_ERR_SIZE;
  }
  void* base = nullptr;
  int st = scratch_address(&base);
  if (st != VP_OK) return st;
  unsigned char* sb = (unsigned char*)base;
  cudaStream_t s = (cudaStream_t)stream;

  StaticTables t{};
  int m[3], oct[3];
  for (int a = 0; a < 3; ++a) {
    m[a] = default_m(g->n[a]);
    oct[a] = m[a] / 2 + 1;
    t.m[a] = m[a];
    t.npass[a] = default_schedule(m[a], t.radix[a]);
    if (t.npass[a] == 0 || m[a] > kStaticMaxM) return VP_ERR_SIZE;
    t.tw[a] = (float2*)(sb + kOffTw) + (size_t)a * kStaticMaxM;
    t.pos[a] = (int*)(sb + kOffPos) + (size_t)a * kStaticMaxM;
    t.fold[a] = (int*)(sb + kOffFold) + (size_t)a * kStaticMaxM;
  }
  t.tiles = (int*)(sb + kOffTiles);
  t.ox = oct[0];
  t.oy = oct[1];
  t.ntiles = (oct[0] * oct[1] + 3) / 4;

  vp::AxisDesc ax[3];
  for (int a = 0; a < 3; ++a) {
    ax[a] = vp::AxisDesc{};
    ax[a].L = m[a];
    ax[a].npass = t.npass[a];
    int lp = m[a];
    for (int i = 0; i < vp::kMaxPass; ++i) {
      ax[a].radix[i] = t.radix[a][i];
      ax[a].lp[i] = i < t.npass[a] ? lp : 0;
      ax[a].magic[i] = 0;
      if (i < t.npass[a]) {
        const unsigned long long sp = (unsigned long long)(lp / t.radix[a][i]);
        ax[a].magic[i] = sp > 1 ? (unsigned)((1ULL << 32) / sp + 1) : 0u;
        lp /= t.radix[a][i];
      }
    }
    ax[a].tw = t.tw[a];
  }

  const double fn = harmonic_n * f0_hz;
  const double kr = 2.0 * kPi * fn / med->c0;
  const double ki = med->alpha0 * std::pow(fn / 1.0e6, med->eta) / (20.0 * std::log10(std::exp(1.0)));
  const int Nx = g->n[0], Ny = g->n[1], Nz = g->n[2];
  const int Mx = m[0], My = m[1], Mz = m[2];
  float2* cube = (float2*)(sb + kOffCube);
  float2* khat = (float2*)(sb + kOffOct);
  float2* wsA = cube;                              // M_x N_y N_z
  float2* wsB = cube + (size_t)Mx * Ny * Nz;       // M_x M_y N_z
  const long long total = (long long)Mx * My * Mz;

  static_tables_kernel<<<64, 256, 0, s>>>(t);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = vp::launch_kernel_lattice(cube, g->n, m, g->h, kr, ki, s);
  if (e == cudaSuccess) {  // spectrum: x, y column sweeps and the z line sweep, in place
    vp::ColSweep c{};
    c.ax = ax[0];
    c.in = cube;
    c.out = cube;
    c.in_rs = c.out_rs = (long long)My * Mz;
    c.in_os = c.out_os = Mz;
    c.C = Mz;
    c.n_outer = My;
    c.rows_in = c.rows_out = Mx;
    c.in_elems = c.out_elems = total;
    c.scale = 1.0f;
    e = vp::launch_col_sweep(c, vp::kForward, false, s);
  }
  if (e == cudaSuccess) {
    vp::ColSweep c{};
    c.ax = ax[1];
    c.in = cube;
    c.out = cube;
    c.in_rs = c.out_rs = Mz;
    c.in_os = c.out_os = (long long)My * Mz;
    c.C = Mz;
    c.n_outer = Mx;
    c.rows_in = c.rows_out = My;
    c.in_elems = c.out_elems = total;
    c.scale = 1.0f;
    e = vp::launch_col_sweep(c, vp::kForward, false, s);
  }
  if (e == cudaSuccess) {
    vp::LineSweep l{};
    l.ax = ax[2];
    l.data = cube;
    l.nlines = (long long)Mx * My;
    l.ld = Mz;
    l.n_in = l.n_out = Mz;
    l.data_elems = total;
    e = vp::launch_line_sweep(l, vp::kForwardOnly, s);
  }
  if (e == cudaSuccess) e = vp::launch_octant_extract(cube, khat, m, oct, t.pos[0], t.pos[1], t.pos[2], s);
  // the lattice cube is dead from here on: its region becomes the FFT workspace
  if (e == cudaSuccess) {
    vp::ColSweep c{};
    c.ax = ax[0];
    c.in = (const float2*)f;
    c.in_rs = (long long)Ny * Nz;
    c.in_os = Nz;
    c.rows_in = Nx;
    c.out = wsA;
    c.out_rs = (long long)Ny * Nz;
    c.out_os = Nz;
    c.rows_out = Mx;
    c.C = Nz;
    c.n_outer = Ny;
    c.in_elems = (long long)Nx * Ny * Nz;
    c.out_elems = (long long)Mx * Ny * Nz;
    c.scale = 1.0f;
    e = vp::launch_col_sweep(c, vp::kForward, false, s);
  }
  if (e == cudaSuccess) {
    vp::ColSweep c{};
    c.ax = ax[1];
    c.in = wsA;
    c.in_rs = Nz;
    c.in_os = (long long)Ny * Nz;
    c.rows_in = Ny;
    c.out = wsB;
    c.out_rs = Nz;
    c.out_os = (long long)My * Nz;
    c.rows_out = My;
    c.C = Nz;
    c.n_outer = Mx;
    c.in_elems = (long long)Mx * Ny * Nz;
    c.out_elems = (long long)Mx * My * Nz;
    c.scale = 1.0f;
    e = vp::launch_col_sweep(c, vp::kForward, false, s);
  }
  if (e == cudaSuccess) {
    vp::LineSweep l{};
    l.ax = ax[2];
    l.data = wsB;
    l.nlines = t.ntiles;
    l.ld = Nz;
    l.n_in = l.n_out = Nz;
    l.data_elems = (long long)Mx * My * Nz;
    l.khat = khat;
    l.Oz = oct[2];
    l.tiles = t.tiles;
    l.fold_z = t.fold[2];
    e = vp::launch_line_sweep(l, vp::kConv, s);
  }
  if (e == cudaSuccess) {
    vp::ColSweep c{};
    c.ax = ax[1];
    c.in = wsB;
    c.in_rs = Nz;
    c.in_os = (long long)My * Nz;
    c.rows_in = My;
    c.out = wsA;
    c.out_rs = Nz;
    c.out_os = (long long)Ny * Nz;
    c.rows_out = Ny;
    c.C = Nz;
    c.n_outer = Mx;
    c.in_elems = (long long)Mx * My * Nz;
    c.out_elems = (long long)Mx * Ny * Nz;
    c.scale = 1.0f;
    e = vp::launch_col_sweep(c, vp::kInverse, false, s);
  }
  if (e == cudaSuccess) {
    vp::ColSweep c{};
    c.ax = ax[0];
    c.in = wsA;
    c.in_rs = (long long)Ny * Nz;
    c.in_os = Nz;
    c.rows_in = Mx;
    c.out = (float2*)u;
    c.out_rs = (long long)Ny * Nz;
    c.out_os = Nz;
    c.rows_out = Nx;
    c.C = Nz;
    c.n_outer = Ny;
    c.in_elems = (long long)Mx * Ny * Nz;
    c.out_elems = (long long)Nx * Ny * Nz;
    c.scale = (float)(1.0 / ((double)Mx * My * Mz));
    e = vp::launch_col_sweep(c, vp::kInverse, false, s);
  }
  return e == cudaSuccess ? VP_OK : VP_ERR_CUDA;
}
