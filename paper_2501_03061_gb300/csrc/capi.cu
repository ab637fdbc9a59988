// The exported C ABI (include/ptim.h): argument checks, context, error conversion.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "trace.h"

namespace pt {

std::atomic<long long> g_launches{0};

void fail(pt_status code, const std::string& msg) { throw Error{code, msg}; }

void check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  if (e == cudaErrorMemoryAllocation) fail(PT_OOM, std::string(what) + ": " + cudaGetErrorString(e));
  fail(PT_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void require_aligned(const void* p, const char* what) {
  if (!p) fail(PT_INVALID_ARG, std::string(what) + " is NULL");
  if (reinterpret_cast<uintptr_t>(p) % 16 != 0) fail(PT_INVALID_ARG, std::string(what) + " is not 16-byte aligned");
}

}  // namespace pt

void* pt_ctx::get(const std::string& name, size_t bytes) {
  auto it = bufs.find(name);
  if (it != bufs.end() && it->second.bytes >= bytes) return it->second.ptr;
  if (it != bufs.end()) {
    pt::check_cuda(cudaDeviceSynchronize(), "workspace resize");
    cudaFree(it->second.ptr);
    held -= it->second.bytes;
    bufs.erase(it);
  }
  bytes = std::max<size_t>(bytes, 256);
  if (budget && held + bytes > budget)
    pt::fail(PT_OOM, "workspace '" + name + "' of " + std::to_string(bytes) + " bytes exceeds the HBM budget");
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    pt::fail(PT_OOM, "cudaMalloc of workspace '" + name + "' (" + std::to_string(bytes) + " bytes) failed");
  }
  bufs[name] = pt::DevBuf{p, bytes};
  held += bytes;
  return p;
}

void pt_ctx::release_all() {
  cudaDeviceSynchronize();
  for (auto& kv : bufs) cudaFree(kv.second.ptr);
  bufs.clear();
  held = 0;
  tc_err_clean = false;
  ptim_q_n = 0;
  ptim_warm_valid = false;  // "ptim_xi" is freed
  // captured graphs hold pointers into the freed workspace
  for (auto it = caches.begin(); it != caches.end();) {
    if (it->first.rfind("graph:", 0) == 0) it = caches.erase(it);
    else ++it;
  }
}

namespace {

// every entry point: an NVTX range named after it, C++ errors turned into status codes
template <class F>
pt_status guarded(const char* entry, pt_ctx* ctx, F&& f) {
  pt::TraceRange range(entry);
  try {
    pt_status s = f();
    if (ctx && s == PT_OK) ctx->err.clear();
    return s;
  } catch (const pt::Error& e) {
    if (ctx) ctx->err = e.msg;
    return e.code;
  } catch (const std::exception& e) {
    if (ctx) ctx->err = e.what();
    return PT_CUDA;
  }
}

void set_device(pt_ctx* ctx) { pt::check_cuda(cudaSetDevice(ctx->device), "cudaSetDevice"); }

// contraction engine for this call: TF32 form on single-product tensor cores, BF16 form on bf16
// tensor cores (packed operands), FP32 form on 3xTF32 tensor cores when the context option asks
// for it, CUDA cores otherwise
void set_engine(pt_ctx* ctx, pt_precision prec) {
  ctx->active_tc = (prec == PT_FP32_TC_TF32) ? 2 : ((prec == PT_FP32 && ctx->tc_gram) ? 1 : 0);
  ctx->bf16_requested = (prec == PT_FP32_TC_BF16);
}

void check_common(pt_ctx* ctx, const pt_grid* grid, pt_precision prec) {
  if (!ctx) pt::fail(PT_INVALID_ARG, "context is NULL");
  pt::validate_grid(grid);
  if (prec < PT_FP64 || prec > PT_FP32_TC_BF16) pt::fail(PT_INVALID_ARG, "unknown precision");
}

// orbital counts: positive and small enough that N*N fits the kernels' 32-bit indices
void check_count(int n, const char* what) {
  if (n <= 0 || n > PT_MAX_ORBITALS)
    pt::fail(PT_INVALID_ARG, std::string(what) + " must be in 1.." + std::to_string(PT_MAX_ORBITALS));
}

void check_kernel(const pt_kernel* k) {
  if (!k) pt::fail(PT_INVALID_ARG, "kernel is NULL");
  if (k->type != 0 && k->type != 1) pt::fail(PT_INVALID_ARG, "kernel type must be 0 or 1");
  if (k->type == 1 && !(k->mu > 0)) pt::fail(PT_INVALID_ARG, "screened kernel needs mu > 0");
}

}  // namespace

extern "C" {

pt_status pt_create(pt_ctx** out, int device, size_t hbm_budget) {
  if (!out) return PT_INVALID_ARG;
  *out = nullptr;
  auto* ctx = new pt_ctx();
  pt_status s = guarded(__func__, ctx, [&]() -> pt_status {
    int n = 0;
    pt::check_cuda(cudaGetDeviceCount(&n), "cudaGetDeviceCount");
    if (device < 0 || device >= n) pt::fail(PT_INVALID_ARG, "no such CUDA device");
    ctx->device = device;
    set_device(ctx);
    cudaDeviceProp prop;
    pt::check_cuda(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");
    ctx->num_sms = prop.multiProcessorCount;
    ctx->max_smem_optin = prop.sharedMemPerBlockOptin;
    size_t free_b = 0, total_b = 0;
    pt::check_cuda(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
    ctx->budget = hbm_budget ? hbm_budget : size_t(0.9 * double(free_b));
    pt::check_cuda(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    return PT_OK;
  });
  if (s != PT_OK) {
    delete ctx;
    return s;
  }
  *out = ctx;
  return PT_OK;
}

void pt_destroy(pt_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  ctx->release_all();
  ctx->caches.clear();
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  for (cudaStream_t s : ctx->side_streams) cudaStreamDestroy(s);
  delete ctx;
}

const char* pt_last_error(const pt_ctx* ctx) { return ctx ? ctx->err.c_str() : "context is NULL"; }

size_t pt_workspace_bytes(const pt_ctx* ctx) { return ctx ? ctx->held : 0; }

pt_status pt_trim(pt_ctx* ctx) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    if (!ctx) pt::fail(PT_INVALID_ARG, "context is NULL");
    set_device(ctx);
    ctx->release_all();
    return PT_OK;
  });
}

pt_status pt_set_option(pt_ctx* ctx, const char* key, double value) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    if (!ctx || !key) pt::fail(PT_INVALID_ARG, "context or key is NULL");
    if (std::string(key) == "fft_threads") {
      if (!(value == 128.0 || value == 256.0 || value == 512.0)) pt::fail(PT_INVALID_ARG, "fft_threads is 128, 256 or 512");
      ctx->fft_threads = int(value);
      return PT_OK;
    }
    if (std::string(key) == "batch_streams") {
      if (!(value >= 1.0 && value <= 16.0)) pt::fail(PT_INVALID_ARG, "batch_streams must be in [1, 16]");
      ctx->batch_streams = int(value);
      return PT_OK;
    }
    if (std::string(key) == "graphs" || std::string(key) == "autotune") {
      (std::string(key) == "graphs" ? ctx->use_graphs : ctx->autotune) = value != 0.0 ? 1 : 0;
      return PT_OK;
    }
    if (std::string(key) == "ptim_inner_kappa" || std::string(key) == "ptim_inner_cap") {
      if (!(value >= 0.0) || value > 1.0) pt::fail(PT_INVALID_ARG, std::string(key) + " must be in [0, 1]");
      (std::string(key) == "ptim_inner_kappa" ? ctx->ptim_inner_kappa : ctx->ptim_inner_cap) = value;
      return PT_OK;
    }
    if (std::string(key) == "ptim_precond") {
      ctx->ptim_precond = value != 0.0 ? 1 : 0;
      return PT_OK;
    }
    if (std::string(key) == "ptim_sinv_mixed") {
      ctx->ptim_sinv_mixed = value != 0.0 ? 1 : 0;
      return PT_OK;
    }
    if (std::string(key) == "ptim_pw") {
      ctx->ptim_pw = value != 0.0 ? 1 : 0;
      return PT_OK;
    }
    if (std::string(key) == "ptim_sinv_series") {
      if (!(value == 0.0 || value == 1.0 || value == 2.0)) pt::fail(PT_INVALID_ARG, "ptim_sinv_series must be 0, 1 or 2");
      ctx->ptim_sinv_series = int(value);
      return PT_OK;
    }
    if (std::string(key) == "ptim_ace_warm") {
      ctx->ptim_ace_warm = value != 0.0 ? 1 : 0;
      return PT_OK;
    }
    if (std::string(key) == "exchange64_engine") {
      if (!(value == 0.0 || value == 1.0 || value == 2.0 || value == 3.0))
        pt::fail(PT_INVALID_ARG, "exchange64_engine is 0, 1, 2 or 3");
      ctx->exchange64_engine = int(value);
      return PT_OK;
    }
    if (std::string(key) == "exchange64p_tile" || std::string(key) == "exchange64p_ring" ||
        std::string(key) == "exchange64p_lag") {
      if (!(value >= 1.0 && value <= 1024.0)) pt::fail(PT_INVALID_ARG, std::string(key) + " must be in [1, 1024]");
      (std::string(key) == "exchange64p_tile" ? ctx->x64p_tile
                                              : (std::string(key) == "exchange64p_ring" ? ctx->x64p_ring
                                                                                        : ctx->x64p_lag)) = int(value);
      return PT_OK;
    }
    if (std::string(key) == "tc_period") {
      if (value < 1 || value > 64) pt::fail(PT_INVALID_ARG, "tc_period must be in [1, 64]");
      ctx->tc_period = int(value);
      return PT_OK;
    }
    if (std::string(key) == "tc_gram_wide") {
      ctx->tc_gram_wide = value != 0.0 ? 1 : 0;
      return PT_OK;
    }
    if (std::string(key) == "tc_gram") {
      ctx->tc_gram = value != 0.0 ? 1 : 0;
      return PT_OK;
    }
    if (std::string(key) == "scratch_bytes") {
      if (!(value >= 1.0)) pt::fail(PT_INVALID_ARG, "scratch_bytes must be >= 1");
      ctx->scratch_budget = size_t(value);
      return PT_OK;
    }
    if (std::string(key) == "exchange64_scratch_bytes") {
      if (!(value >= 1.0)) pt::fail(PT_INVALID_ARG, "exchange64_scratch_bytes must be >= 1");
      ctx->tma64_budget = size_t(value);
      return PT_OK;
    }
    pt::fail(PT_INVALID_ARG, std::string("unknown option ") + key);
  });
}

pt_status pt_apply_exchange(pt_ctx* ctx, const void* src, const double* occ, int N, const void* tgt, int M,
                            void* out, const pt_grid* grid, const pt_kernel* kernel, pt_precision prec,
                            void* stream) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    check_common(ctx, grid, prec);
    check_kernel(kernel);
    check_count(N, "N");
    if (tgt == nullptr) M = N;
    check_count(M, "M");
    pt::require_aligned(src, "src");
    pt::require_aligned(out, "out");
    if (!occ) pt::fail(PT_INVALID_ARG, "occ is NULL");
    if (tgt) pt::require_aligned(tgt, "tgt");
    if (out == src || (tgt && out == tgt)) pt::fail(PT_INVALID_ARG, "out must not alias src or tgt");
    set_device(ctx);
    set_engine(ctx, prec);
    pt::exchange(ctx, src, occ, N, tgt, M, out, *grid, *kernel, prec, static_cast<cudaStream_t>(stream));
    return PT_OK;
  });
}

pt_status pt_apply_exchange_mixed(pt_ctx* ctx, const void* phi, const void* sigma, int N, const void* tgt, int M,
                                  void* out, const pt_grid* grid, const pt_kernel* kernel, pt_precision prec,
                                  long long* pair_ffts, void* stream) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    check_common(ctx, grid, prec);
    check_kernel(kernel);
    check_count(N, "N");
    if (tgt == nullptr) M = N;
    check_count(M, "M");
    pt::require_aligned(phi, "phi");
    pt::require_aligned(sigma, "sigma");
    pt::require_aligned(out, "out");
    if (tgt) pt::require_aligned(tgt, "tgt");
    if (out == phi || (tgt && out == tgt)) pt::fail(PT_INVALID_ARG, "out must not alias phi or tgt");
    set_device(ctx);
    set_engine(ctx, prec);
    const long long n = pt::exchange_mixed(ctx, phi, static_cast<const c128*>(sigma), N, tgt, M, out, *grid, *kernel,
                                           prec, static_cast<cudaStream_t>(stream));
    if (pair_ffts) *pair_ffts = n;
    return PT_OK;
  });
}

pt_status pt_apply_exchange_batched(pt_ctx* ctx, const pt_exchange_item* items, int count, pt_precision prec,
                                    long long* pair_ffts, size_t* graph_nodes, void* stream) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    if (!ctx) pt::fail(PT_INVALID_ARG, "context is NULL");
    if (count <= 0 || !items) pt::fail(PT_INVALID_ARG, "no items");
    if (prec < PT_FP64 || prec > PT_FP32_TC_BF16) pt::fail(PT_INVALID_ARG, "unknown precision");
    for (int k = 0; k < count; ++k) {
      const pt_exchange_item& it = items[k];
      const std::string w = "item " + std::to_string(k) + ": ";
      try {
        pt::validate_grid(&it.grid);
        check_kernel(&it.kernel);
      } catch (const pt::Error& e) {
        pt::fail(e.code, w + e.msg);
      }
      if (it.N <= 0 || it.N > PT_MAX_ORBITALS || (it.tgt && (it.M <= 0 || it.M > PT_MAX_ORBITALS)))
        pt::fail(PT_INVALID_ARG, w + "N and M must be in 1.." + std::to_string(PT_MAX_ORBITALS));
      if (!it.occ) pt::fail(PT_INVALID_ARG, w + "occ is NULL");
      pt::require_aligned(it.src, "src");
      pt::require_aligned(it.out, "out");
      if (it.tgt) pt::require_aligned(it.tgt, "tgt");
      if (it.out == it.src || (it.tgt && it.out == it.tgt))
        pt::fail(PT_INVALID_ARG, w + "out must not alias src or tgt");
    }
    set_device(ctx);
    const long long n = pt::exchange_batched(ctx, items, count, prec, static_cast<cudaStream_t>(stream), graph_nodes);
    if (pair_ffts) *pair_ffts = n;
    return PT_OK;
  });
}

pt_status pt_build_ace_from(pt_ctx* ctx, const void* W, const void* phi, int N, const pt_grid* grid,
                            pt_precision prec, pt_ace** ace, void* stream) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    check_common(ctx, grid, prec);
    if (!ace) pt::fail(PT_INVALID_ARG, "ace is NULL");
    *ace = nullptr;
    check_count(N, "N");
    pt::require_aligned(W, "W");
    pt::require_aligned(phi, "phi");
    set_device(ctx);
    set_engine(ctx, prec);
    auto* a = new pt_ace();
    a->ctx = ctx;
    a->N = N;
    a->grid = *grid;
    a->prec = prec;
    a->bytes = pt::ng_of(*grid) * N * pt::elem_bytes(prec);
    cudaError_t e = cudaMalloc(&a->xi, a->bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete a;
      pt::fail(PT_OOM, "cannot allocate the ACE vectors");
    }
    try {
      pt::ace_from_w(ctx, W, phi, N, *grid, prec, a->xi, static_cast<cudaStream_t>(stream));
      if (ctx->active_tc || ctx->bf16_requested) pt::gram_tc_check(ctx, static_cast<cudaStream_t>(stream));
    } catch (...) {
      cudaFree(a->xi);
      delete a;
      throw;
    }
    *ace = a;
    return PT_OK;
  });
}

pt_status pt_build_ace(pt_ctx* ctx, const void* phi, const double* occ, int N, const pt_grid* grid,
                       const pt_kernel* kernel, pt_precision prec, pt_ace** ace, void* stream) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    check_common(ctx, grid, prec);
    check_kernel(kernel);
    if (!ace) pt::fail(PT_INVALID_ARG, "ace is NULL");
    check_count(N, "N");
    pt::require_aligned(phi, "phi");
    if (!occ) pt::fail(PT_INVALID_ARG, "occ is NULL");
    set_device(ctx);
    const size_t bytes = pt::ng_of(*grid) * N * pt::elem_bytes(prec);
    void* W = ctx->get("build_ace_W", bytes);
    pt::exchange(ctx, phi, occ, N, nullptr, N, W, *grid, *kernel, prec, static_cast<cudaStream_t>(stream));
    pt_status s = pt_build_ace_from(ctx, W, phi, N, grid, prec, ace, stream);
    if (s != PT_OK) pt::fail(s, ctx->err);
    return PT_OK;
  });
}

pt_status pt_overlap(pt_ctx* ctx, const void* A, int N1, const void* B, int N2, const pt_grid* grid,
                     pt_precision prec, void* C, void* stream) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    check_common(ctx, grid, prec);
    check_count(N1, "N1");
    check_count(N2, "N2");
    pt::require_aligned(A, "A");
    pt::require_aligned(B, "B");
    pt::require_aligned(C, "C");
    set_device(ctx);
    set_engine(ctx, prec);
    auto st = static_cast<cudaStream_t>(stream);
    const size_t ng = pt::ng_of(*grid);
    const double dV = pt::dv_of(*grid);
    auto* Cm = static_cast<c128*>(C);
    const bool herm = (A == B && N1 == N2);  // Hermitian result: compute one triangle of tiles
    if (prec == PT_FP64)
      pt::gram<double>(ctx, static_cast<const c128*>(A), static_cast<const c128*>(B), N1, N2, ng, dV, Cm, st, herm);
    else
      pt::gram<float>(ctx, static_cast<const c64*>(A), static_cast<const c64*>(B), N1, N2, ng, dV, Cm, st, herm);
    if (ctx->active_tc || ctx->bf16_requested) pt::gram_tc_check(ctx, st);
    return PT_OK;
  });
}

pt_status pt_rotate(pt_ctx* ctx, const void* A, int N1, const void* B, int N2, const pt_grid* grid,
                    pt_precision prec, void* out, void* stream) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    check_common(ctx, grid, prec);
    check_count(N1, "N1");
    check_count(N2, "N2");
    pt::require_aligned(A, "A");
    pt::require_aligned(B, "B");
    pt::require_aligned(out, "out");
    const size_t ng = pt::ng_of(*grid), eb = pt::elem_bytes(prec);
    const char* a0 = static_cast<const char*>(A);
    const char* o0 = static_cast<const char*>(out);
    if (o0 < a0 + ng * N1 * eb && a0 < o0 + ng * N2 * eb) pt::fail(PT_INVALID_ARG, "out overlaps A");
    set_device(ctx);
    set_engine(ctx, prec);
    auto st = static_cast<cudaStream_t>(stream);
    const auto* Bm = static_cast<const c128*>(B);
    if (prec == PT_FP64)
      pt::rotate<double>(ctx, static_cast<const c128*>(A), Bm, N2, N1, N2, ng, c128{1, 0}, nullptr, 0,
                         static_cast<c128*>(out), st);
    else
      pt::rotate<float>(ctx, static_cast<const c64*>(A), Bm, N2, N1, N2, ng, c128{1, 0}, nullptr, 0,
                        static_cast<c64*>(out), st);
    if (ctx->active_tc || ctx->bf16_requested) pt::gram_tc_check(ctx, st);
    return PT_OK;
  });
}

pt_status pt_apply_ace(pt_ctx* ctx, const pt_ace* ace, const void* psi, int M, void* out, void* stream) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    if (!ctx || !ace) pt::fail(PT_INVALID_ARG, "context or ACE is NULL");
    check_count(M, "M");
    pt::require_aligned(psi, "psi");
    pt::require_aligned(out, "out");
    if (out == psi) pt::fail(PT_INVALID_ARG, "out must not alias psi");
    set_device(ctx);
    set_engine(ctx, ace->prec);
    pt::ace_apply(ctx, ace->xi, ace->N, psi, M, out, ace->grid, ace->prec, static_cast<cudaStream_t>(stream));
    if (ctx->active_tc || ctx->bf16_requested) pt::gram_tc_check(ctx, static_cast<cudaStream_t>(stream));
    return PT_OK;
  });
}

pt_status pt_ace_get_xi(const pt_ace* ace, void* xi_out, void* stream) {
  if (!ace || !xi_out) return PT_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(xi_out, ace->xi, ace->bytes, cudaMemcpyDeviceToDevice,
                                  static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PT_OK : PT_CUDA;
}

void pt_ace_destroy(pt_ace* ace) {
  if (!ace) return;
  cudaFree(ace->xi);
  delete ace;
}

pt_status pt_apply_H(pt_ctx* ctx, const void* psi, int M, void* out, const double* vloc, const pt_ace* ace,
                     double alpha, double ecut, const double* A, const pt_grid* grid, pt_precision prec,
                     void* stream) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    check_common(ctx, grid, prec);
    check_count(M, "M");
    pt::require_aligned(psi, "psi");
    pt::require_aligned(out, "out");
    if (!vloc) pt::fail(PT_INVALID_ARG, "vloc is NULL");
    if (out == psi) pt::fail(PT_INVALID_ARG, "out must not alias psi");
    if (ace && (ace->prec != prec || ace->grid.nx != grid->nx || ace->grid.ny != grid->ny || ace->grid.nz != grid->nz))
      pt::fail(PT_INVALID_ARG, "ACE operator does not match the grid or precision");
    set_device(ctx);
    set_engine(ctx, prec);
    auto st = static_cast<cudaStream_t>(stream);
    const void* X = nullptr;
    if (ace) {
      void* buf = ctx->get("apply_H_X", pt::ng_of(*grid) * M * pt::elem_bytes(prec));
      pt::ace_apply(ctx, ace->xi, ace->N, psi, M, buf, *grid, prec, st);
      X = buf;
    }
    pt::apply_h(ctx, psi, M, out, vloc, X, alpha, ecut, *grid, prec, st, A);
    if ((ctx->active_tc || ctx->bf16_requested) && ace) pt::gram_tc_check(ctx, st);
    return PT_OK;
  });
}

pt_status pt_current(pt_ctx* ctx, const void* phi, const void* sigma, int N, const pt_grid* grid, pt_precision prec,
                     const double* A, double spin, double* J, void* stream) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    check_common(ctx, grid, prec);
    check_count(N, "N");
    if (!phi || !sigma || !J) pt::fail(PT_INVALID_ARG, "NULL buffer");
    pt::require_aligned(phi, "phi");
    pt::require_aligned(sigma, "sigma");
    set_device(ctx);
    set_engine(ctx, prec);
    auto st = static_cast<cudaStream_t>(stream);
    pt::current(ctx, phi, static_cast<const c128*>(sigma), N, *grid, prec, A, spin, J, st);
    if (ctx->active_tc || ctx->bf16_requested) pt::gram_tc_check(ctx, st);
    return PT_OK;
  });
}

pt_status pt_density(pt_ctx* ctx, const void* phi, const void* sigma, int N, const pt_grid* grid, pt_precision prec,
                     double spin, double* rho, void* stream) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    check_common(ctx, grid, prec);
    check_count(N, "N");
    if (!phi || !sigma || !rho) pt::fail(PT_INVALID_ARG, "NULL buffer");
    if (!(spin > 0.0)) pt::fail(PT_INVALID_ARG, "spin must be positive");
    pt::require_aligned(phi, "phi");
    pt::require_aligned(sigma, "sigma");
    set_device(ctx);
    set_engine(ctx, prec);
    auto st = static_cast<cudaStream_t>(stream);
    const size_t ng = pt::ng_of(*grid);
    void* chi = ctx->get("density_chi", ng * size_t(N) * pt::elem_bytes(prec));
    if (prec == PT_FP64)
      pt::density<double>(ctx, static_cast<const c128*>(phi), static_cast<const c128*>(sigma), N, ng, spin,
                          static_cast<c128*>(chi), rho, st);
    else
      pt::density<float>(ctx, static_cast<const c64*>(phi), static_cast<const c128*>(sigma), N, ng, spin,
                         static_cast<c64*>(chi), rho, st);
    if (ctx->active_tc || ctx->bf16_requested) pt::gram_tc_check(ctx, st);
    return PT_OK;
  });
}

pt_status pt_hxc_potential(pt_ctx* ctx, const double* rho, const double* vloc, const pt_grid* grid, double* v,
                           double* energies, void* stream) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    if (!ctx) pt::fail(PT_INVALID_ARG, "context is NULL");
    pt::validate_grid(grid);
    if (!rho || !v) pt::fail(PT_INVALID_ARG, "NULL buffer");
    if (v == rho) pt::fail(PT_INVALID_ARG, "v must not alias rho");
    set_device(ctx);
    auto st = static_cast<cudaStream_t>(stream);
    double* part = energies ? static_cast<double*>(ctx->get("hxc_part", 2 * size_t(grid->nz) * sizeof(double)))
                            : nullptr;
    pt::hxc_potential(ctx, rho, vloc, *grid, v, part, st);
    if (energies) {
      std::vector<double> h(2 * size_t(grid->nz));
      PT_CUDA_CHECK(cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      PT_CUDA_CHECK(cudaStreamSynchronize(st));
      double eh = 0.0, exc = 0.0;
      for (int z = 0; z < grid->nz; ++z) {
        eh += h[2 * z];
        exc += h[2 * z + 1];
      }
      const double dv = pt::dv_of(*grid);
      energies[0] = eh * dv;
      energies[1] = exc * dv;
    }
    return PT_OK;
  });
}

pt_status pt_diag_occupations(pt_ctx* ctx, const void* sigma, int N, void* Q, double* d, void* stream) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    if (!ctx) pt::fail(PT_INVALID_ARG, "context is NULL");
    check_count(N, "N");
    if (!sigma || !Q || !d) pt::fail(PT_INVALID_ARG, "NULL buffer");
    pt::require_aligned(sigma, "sigma");
    pt::require_aligned(Q, "Q");
    set_device(ctx);
    pt::heev(ctx, static_cast<const c128*>(sigma), N, static_cast<c128*>(Q), d, static_cast<cudaStream_t>(stream));
    return PT_OK;
  });
}

pt_status pt_ptim_step(pt_ctx* ctx, void* phi, void* sigma, int N, const double* vloc, const pt_grid* grid,
                       const pt_kernel* kernel, const pt_ptim_params* params, pt_precision prec,
                       pt_ptim_stats* stats, void* stream) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    check_common(ctx, grid, prec);
    check_kernel(kernel);
    if (!params) pt::fail(PT_INVALID_ARG, "params is NULL");
    check_count(N, "N");
    pt::require_aligned(phi, "phi");
    pt::require_aligned(sigma, "sigma");
    if (!vloc) pt::fail(PT_INVALID_ARG, "vloc is NULL");
    const pt_ptim_params& P = *params;
    if (!(P.dt > 0) || !(P.tol > 0) || !(P.ecut > 0) || P.max_inner <= 0 || P.max_outer <= 0 || P.anderson_depth <= 0 ||
        P.anderson_depth > 20 || (P.hxc != 0 && P.hxc != 1) || (P.hxc && !(P.spin > 0)))
      pt::fail(PT_INVALID_ARG, "invalid PT-IM parameters");
    set_device(ctx);
    set_engine(ctx, prec);
    pt_status r =
        pt::ptim_step(ctx, phi, sigma, N, vloc, *grid, *kernel, P, prec, stats, static_cast<cudaStream_t>(stream));
    if (ctx->active_tc || ctx->bf16_requested) pt::gram_tc_check(ctx, static_cast<cudaStream_t>(stream));
    return r;
  });
}

size_t pt_ptim_footprint(int N, const pt_grid* grid, pt_precision prec, int anderson_depth) {
  if (!grid || N <= 0 || N > PT_MAX_ORBITALS) return 0;
  const size_t ng = pt::ng_of(*grid);
  const size_t es = pt::elem_bytes(prec);
  const size_t field = ng * es;
  const size_t block = field * size_t(N);
  const int depth = anderson_depth < 1 ? 1 : (anderson_depth > 20 ? 20 : anderson_depth);
  const size_t budget = size_t(512) << 20;  // default scratch_bytes of a context
  size_t B = size_t(std::floor(std::sqrt(double(std::max<size_t>(1, budget / field)))));
  B = std::max<size_t>(1, std::min<size_t>(B, size_t(N)));
  const bool tma64 = grid->nx == 64 && grid->ny == 64 && grid->nz == 64 && prec != PT_FP64;
  if (tma64) {
    const size_t b64 = size_t(std::floor(std::sqrt(double((size_t(512) << 20) / field))));  // default tma64_budget
    B = std::max<size_t>(1, std::min<size_t>({b64, size_t(N), size_t(pt::kExchange64MaxTile)}));
  }
  const size_t exch = (tma64 ? 4 : 1) * B * B * field;
  const size_t hscr = 2 * std::max<size_t>(1, std::min<size_t>(size_t(N), budget / (2 * field))) * field;
  const size_t nn = size_t(N) * N * sizeof(double) * 2;
  const size_t gram_parts = size_t(4 * 160 + 64) * nn;  // split partials, bounded by 4 waves of tiles
  const size_t blocks = (12 + 2 * size_t(depth)) * block;
  // N x N matrices: the step's named ones, the eigensolver's and the sigma half of the Anderson ring
  const size_t small = (24 + 2 * size_t(depth)) * nn + (size_t(64) << 20);
  const size_t hxc = 4 * ng * sizeof(double);  // rho, total potential, FFT scratch (params.hxc = 1)
  return blocks + exch + hscr + std::min(gram_parts, size_t(8) * block) + small + hxc;
}

const char* pt_version(void) { return "ptim-gb300 0.1 (sm_103a)"; }

long long pt_kernel_launches(void) { return pt::g_launches.load(); }

pt_status pt_alu_peaks(pt_ctx* ctx, double* fp32_tflops, double* fp64_tflops, void* stream) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    if (!ctx || !fp32_tflops || !fp64_tflops) pt::fail(PT_INVALID_ARG, "context or output is NULL");
    set_device(ctx);
    pt::alu_peaks(ctx, fp32_tflops, fp64_tflops, static_cast<cudaStream_t>(stream));
    return PT_OK;
  });
}

pt_status pt_selftest_wait(pt_ctx* ctx, int arrive, double timeout_s, void* stream) {
  return guarded(__func__, ctx, [&]() -> pt_status {
    if (!ctx) pt::fail(PT_INVALID_ARG, "context is NULL");
    if (arrive != 0 && arrive != 1) pt::fail(PT_INVALID_ARG, "arrive must be 0 or 1");
    if (!(timeout_s > 0.0) || timeout_s > 2.0) pt::fail(PT_INVALID_ARG, "timeout_s must be in (0, 2]");
    set_device(ctx);
    pt::wait_selftest(ctx, arrive, timeout_s, static_cast<cudaStream_t>(stream));
    return PT_OK;
  });
}

}  // extern "C"
