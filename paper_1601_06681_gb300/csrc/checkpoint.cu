// Checkpoint/resume of a context's stepping state, and the inner-sweep autotuner.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ehdg_internal.h"

using namespace ehdg;


// the device arrays a checkpoint carries, in file order
std::vector<std::pair<void*, size_t>> ehdg::state_arrays(Ctx& c) {
  const size_t state = sizeof(double) * (size_t)c.n * c.nel;
  const size_t trace = sizeof(double) * (size_t)c.Nqf * c.nface;
  return {{c.u, state},      {c.uhat, trace},       {c.uhat_n, trace}, {c.gb, trace},
          {c.gb_old, trace}, {c.force, state},      {c.force_old, state},
          {c.warm, sizeof(int)}};
}

namespace {

constexpr uint32_t kMagic = 0x47444845u;   // "EHDG"
constexpr uint32_t kVersion = 2;   // 2: the warm-start flag joins the state

struct Crc32Table {
  uint32_t t[256];
  Crc32Table() {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int k = 0; k < 8; ++k) c = (c & 1) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
      t[i] = c;
    }
  }
};

uint32_t crc32_update(uint32_t crc, const void* data, size_t n) {
  // a function-local static is initialised exactly once, thread-safely, so
  // checkpoints of different contexts may be written from several threads
  static const Crc32Table table;
  const unsigned char* p = static_cast<const unsigned char*>(data);
  crc = ~crc;
  for (size_t i = 0; i < n; ++i) crc = table.t[(crc ^ p[i]) & 0xFFu] ^ (crc >> 8);
  return ~crc;
}

uint64_t fnv1a(uint64_t h, const void* data, size_t n) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

struct Header {
  uint32_t magic, version;
  int32_t dim, p, nf, Np, q, Nqf, scheme, pde, have_force, pad;
  int64_t nel, nface;
  uint64_t config_hash;
  uint64_t payload_bytes;
};

uint64_t config_hash(const Ctx& c) {
  uint64_t h = 1469598103934665603ull;
  h = fnv1a(h, c.elem_lo.data(), sizeof(double) * c.elem_lo.size());
  h = fnv1a(h, c.elem_h.data(), sizeof(double) * c.elem_h.size());
  h = fnv1a(h, c.face_elem_h.data(), sizeof(int64_t) * c.face_elem_h.size());
  h = fnv1a(h, &c.dt, sizeof(double));
  h = fnv1a(h, &c.Phi, sizeof(double));
  const double src[4] = {c.cor_f0, c.cor_beta, c.cor_ym, c.friction};
  h = fnv1a(h, src, sizeof(src));
  h = fnv1a(h, c.beta_const, sizeof(double) * 3);
  // the velocity field of a per-node velocity (beta_const is zero then)
  const int vb = c.variable_beta ? 1 : 0;
  h = fnv1a(h, &vb, sizeof(vb));
  h = fnv1a(h, &c.beta_nodes_hash, sizeof(c.beta_nodes_hash));
  return h;
}

ehdg_status io_fail(ehdg_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

}  // namespace

extern "C" ehdg_status ehdg_save(ehdg_ctx h, const char* path) {
  if (!h || !path) return io_fail(EHDG_ERR_INVALID, "NULL argument");
  Ctx& c = h->c;
  if (cudaStreamSynchronize(c.stream) != cudaSuccess)
    return io_fail(EHDG_ERR_CUDA, "stream synchronisation failed");
  auto arrays = state_arrays(c);
  Header hd{};
  hd.magic = kMagic;
  hd.version = kVersion;
  hd.dim = c.dim;
  hd.p = c.p;
  hd.nf = c.nf;
  hd.Np = c.Np;
  hd.q = c.q;
  hd.Nqf = c.Nqf;
  hd.scheme = c.scheme;
  hd.pde = c.pde;
  hd.have_force = c.have_force ? 1 : 0;
  hd.nel = c.nel;
  hd.nface = c.nface;
  hd.config_hash = config_hash(c);
  for (auto& a : arrays) hd.payload_bytes += a.second;
  FILE* f = std::fopen(path, "wb");
  if (!f) return io_fail(EHDG_ERR_INVALID, std::string("cannot open ") + path);
  bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1;
  uint32_t crc = 0;
  std::vector<char> buf;
  for (auto& a : arrays) {
    if (!ok) break;
    buf.resize(a.second);
    if (cudaMemcpy(buf.data(), a.first, a.second, cudaMemcpyDeviceToHost) != cudaSuccess) {
      std::fclose(f);
      return io_fail(EHDG_ERR_CUDA, "device read failed");
    }
    crc = crc32_update(crc, buf.data(), buf.size());
    ok = std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
  }
  ok = ok && std::fwrite(&crc, sizeof(crc), 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? EHDG_OK : io_fail(EHDG_ERR_INVALID, std::string("write failed: ") + path);
}

extern "C" ehdg_status ehdg_load(ehdg_ctx h, const char* path) {
  if (!h || !path) return io_fail(EHDG_ERR_INVALID, "NULL argument");
  Ctx& c = h->c;
  FILE* f = std::fopen(path, "rb");
  if (!f) return io_fail(EHDG_ERR_INVALID, std::string("cannot open ") + path);
  Header hd{};
  auto arrays = state_arrays(c);
  uint64_t payload = 0;
  for (auto& a : arrays) payload += a.second;
  if (std::fread(&hd, sizeof(hd), 1, f) != 1 || hd.magic != kMagic || hd.version != kVersion) {
    std::fclose(f);
    return io_fail(EHDG_ERR_INVALID, "not an eHDG checkpoint of this version");
  }
  if (hd.dim != c.dim || hd.p != c.p || hd.nf != c.nf || hd.Np != c.Np || hd.q != c.q ||
      hd.Nqf != c.Nqf || hd.scheme != (int)c.scheme || hd.pde != (int)c.pde || hd.nel != c.nel ||
      hd.nface != c.nface || hd.payload_bytes != payload || hd.config_hash != config_hash(c)) {
    std::fclose(f);
    return io_fail(EHDG_ERR_INVALID, "checkpoint belongs to a different mesh or problem");
  }
  std::vector<std::vector<char>> bufs(arrays.size());
  uint32_t crc = 0;
  for (size_t i = 0; i < arrays.size(); ++i) {
    bufs[i].resize(arrays[i].second);
    if (std::fread(bufs[i].data(), 1, bufs[i].size(), f) != bufs[i].size()) {
      std::fclose(f);
      return io_fail(EHDG_ERR_INVALID, "truncated checkpoint");
    }
    crc = crc32_update(crc, bufs[i].data(), bufs[i].size());
  }
  uint32_t stored = 0;
  const bool got = std::fread(&stored, sizeof(stored), 1, f) == 1;
  std::fclose(f);
  if (!got || stored != crc) return io_fail(EHDG_ERR_INVALID, "checkpoint CRC mismatch");
  if (cudaStreamSynchronize(c.stream) != cudaSuccess)
    return io_fail(EHDG_ERR_CUDA, "stream synchronisation failed");
  for (size_t i = 0; i < arrays.size(); ++i)
    if (cudaMemcpy(arrays[i].first, bufs[i].data(), bufs[i].size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return io_fail(EHDG_ERR_CUDA, "device write failed");
  c.have_force = hd.have_force != 0;
  return EHDG_OK;
}

namespace {

// Time one implicit step from the current state under each of n variants
// (apply(k) configures variant k), restoring the state after every step;
// ms[k] is the second of two steps (the first also captures the step graph),
// or 1e300 when apply(k) declines the variant. The state is left as it was.
template <class Apply>
ehdg_status time_step_variants(ehdg_ctx h, int n, Apply apply, double* ms) {
  Ctx& c = h->c;
  auto arrays = state_arrays(c);
  std::vector<void*> snap(arrays.size(), nullptr);
  auto free_snap = [&]() {
    for (void* p : snap)
      if (p) cudaFree(p);
  };
  for (size_t i = 0; i < arrays.size(); ++i) {
    if (cudaMalloc(&snap[i], arrays[i].second) != cudaSuccess ||
        cudaMemcpyAsync(snap[i], arrays[i].first, arrays[i].second, cudaMemcpyDeviceToDevice,
                        c.stream) != cudaSuccess) {
      free_snap();
      return io_fail(EHDG_ERR_OOM, "autotune snapshot failed");
    }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  ehdg_status st = EHDG_OK;
  for (int k = 0; k < n; ++k) {
    ms[k] = 1e300;
    if (st != EHDG_OK || !apply(k)) continue;
    if (c.gexec) {
      cudaGraphExecDestroy(c.gexec);
      c.gexec = nullptr;
    }
    if (c.graph) {
      cudaGraphDestroy(c.graph);
      c.graph = nullptr;
    }
    int iters = 0;
    for (int rep = 0; rep < 2 && st == EHDG_OK; ++rep) {
      cudaEventRecord(e0, c.stream);
      st = ehdg_step(h, &iters, nullptr);
      cudaEventRecord(e1, c.stream);
      cudaEventSynchronize(e1);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep == 1) ms[k] = t;
      for (size_t i = 0; i < arrays.size(); ++i)
        cudaMemcpyAsync(arrays[i].first, snap[i], arrays[i].second, cudaMemcpyDeviceToDevice,
                        c.stream);
    }
  }
  cudaStreamSynchronize(c.stream);
  free_snap();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (c.gexec) {
    cudaGraphExecDestroy(c.gexec);
    c.gexec = nullptr;
  }
  if (c.graph) {
    cudaGraphDestroy(c.graph);
    c.graph = nullptr;
  }
  return st;
}

}  // namespace

extern "C" ehdg_status ehdg_autotune_inner_sweeps(ehdg_ctx h, const int* cands, int n, int* best,
                                                  double* best_ms) {
  if (!h || !cands || n < 1) return io_fail(EHDG_ERR_INVALID, "bad argument");
  Ctx& c = h->c;
  if (!c.mixed) return io_fail(EHDG_ERR_INVALID, "the context is not mixed precision");
  const int saved = c.inner_sweeps;
  std::vector<double> ms((size_t)n);
  const ehdg_status st = time_step_variants(
      h, n,
      [&](int k) {
        if (cands[k] < 1 || cands[k] > 64) return false;
        c.inner_sweeps = cands[k];
        return true;
      },
      ms.data());
  int best_m = saved;
  double best_t = 1e300;
  for (int k = 0; k < n; ++k)
    if (ms[k] < best_t) {
      best_t = ms[k];
      best_m = cands[k];
    }
  c.inner_sweeps = (st == EHDG_OK) ? best_m : saved;
  if (best) *best = c.inner_sweeps;
  if (best_ms) *best_ms = best_t;
  return st;
}

extern "C" ehdg_status ehdg_autotune_fp64_path(ehdg_ctx h, int* tensor_cores, double* ms_dfma,
                                               double* ms_tensor) {
  if (!h) return io_fail(EHDG_ERR_INVALID, "NULL context");
  Ctx& c = h->c;
  if (!c.oz_sweep.img)
    return io_fail(EHDG_ERR_INVALID,
                   "the context has no tensor-core FP64 path (FP64_EMULATED or emulated_outer)");
  const bool saved = c.use_ozaki;
  double ms[2];
  const ehdg_status st = time_step_variants(
      h, 2,
      [&](int k) {
        c.use_ozaki = k == 1;
        return true;
      },
      ms);
  c.use_ozaki = (st == EHDG_OK) ? (ms[1] < ms[0]) : saved;
  ++c.path_gen;
  if (tensor_cores) *tensor_cores = c.use_ozaki ? 1 : 0;
  if (ms_dfma) *ms_dfma = ms[0];
  if (ms_tensor) *ms_tensor = ms[1];
  return st;
}

extern "C" ehdg_status ehdg_autotune_sweep_tile(ehdg_ctx h, const int* cands, int n, int* best,
                                                double* best_ms) {
  if (!h || !cands || n < 1) return io_fail(EHDG_ERR_INVALID, "bad argument");
  Ctx& c = h->c;
  if (c.pde != EHDG_TRANSPORT || c.Hyt || c.use_ozaki || c.use_pe)
    return io_fail(EHDG_ERR_INVALID,
                   "the context's FP64 sweep has no tile choice (it is not the fused transport "
                   "sweep)");
  const int saved = c.sweep_ft;
  std::vector<double> ms((size_t)n);
  const ehdg_status st = time_step_variants(
      h, n,
      [&](int k) {
        if (cands[k] != 2 && cands[k] != 4 && cands[k] != 8) return false;
        c.sweep_ft = cands[k];
        return true;
      },
      ms.data());
  int best_ft = saved;
  double best_t = 1e300;
  for (int k = 0; k < n; ++k)
    if (ms[k] < best_t) {
      best_t = ms[k];
      best_ft = cands[k];
    }
  c.sweep_ft = (st == EHDG_OK) ? best_ft : saved;
  ++c.path_gen;   // a batch recaptures its graph
  if (best) *best = c.sweep_ft;
  if (best_ms) *best_ms = best_t;
  return st;
}
