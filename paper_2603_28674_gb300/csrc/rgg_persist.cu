// Host side of rgg_save / rgg_load.
#include "rgg_host.h"

using namespace rgg;
using namespace rgg_host;

extern "C" {

// ---------------------------------------------------------------------------
// Persistence: rgg_save / rgg_load
// ---------------------------------------------------------------------------
struct SaveHeader {
  char magic[8];
  uint32_t version, L, K, M, Wm;
  float margin;
  uint32_t flags;  // bit 0: regular inner records; bit 1: link-end records
  uint32_t pad;
  uint64_t N, S, n_inner, n_outer;
  uint64_t reserved[3];
};
static_assert(sizeof(SaveHeader) == 96, "save header size");

static const char kSaveMagic[8] = {'R', 'G', 'G', 'S', 'A', 'V', 'E', '1'};
static const size_t kStagingBytes = 64ull << 20;

// 64-bit checksum of a byte stream, eight bytes at a time (xor, multiply by
// an odd constant, fold the high bits down); the stream is fed in pieces.
struct StreamHash {
  uint64_t h = 0x6a09e667f3bcc909ull;
  uint64_t word = 0;
  unsigned fill = 0;
  void mix(uint64_t w) {
    h = (h ^ w) * 0x9e3779b97f4a7c15ull;
    h ^= h >> 29;
  }
  void update(const void* data, size_t n) {
    const unsigned char* p = static_cast<const unsigned char*>(data);
    while (n && fill) {
      word |= (uint64_t)*p++ << (8 * fill);
      --n;
      if (++fill == 8) {
        mix(word);
        word = 0;
        fill = 0;
      }
    }
    for (; n >= 8; n -= 8, p += 8) {
      uint64_t w;
      std::memcpy(&w, p, 8);
      mix(w);
    }
    for (; n; --n) word |= (uint64_t)*p++ << (8 * fill++);
  }
  uint64_t digest() const {
    StreamHash t = *this;
    t.mix(t.word ^ ((uint64_t)t.fill << 56));
    return t.h;
  }
};

struct FileIO {
  FILE* f = nullptr;
  StreamHash hash;
  unsigned char* staging = nullptr;
  bool io_ok = true;
  ~FileIO() {
    if (f) fclose(f);
    if (staging) cudaFreeHost(staging);
  }
  bool put(const void* p, size_t n) {
    if (!io_ok) return false;
    hash.update(p, n);
    io_ok = n == 0 || fwrite(p, 1, n, f) == n;
    return io_ok;
  }
  bool get(void* p, size_t n) {
    if (!io_ok) return false;
    io_ok = n == 0 || fread(p, 1, n, f) == n;
    if (io_ok) hash.update(p, n);
    return io_ok;
  }
};

// Device bytes to the file through the page-locked staging buffer.
static int save_device(FileIO& io, const void* src, size_t bytes, cudaStream_t s) {
  const unsigned char* p = static_cast<const unsigned char*>(src);
  for (size_t off = 0; off < bytes; off += kStagingBytes) {
    const size_t n = std::min(kStagingBytes, bytes - off);
    RGG_CK(cudaMemcpyAsync(io.staging, p + off, n, cudaMemcpyDeviceToHost, s));
    RGG_CK(cudaStreamSynchronize(s));
    if (!io.put(io.staging, n)) return RGG_ERR_IO;
  }
  return RGG_OK;
}

// File bytes to device memory through the staging buffer.  A short read is
// a truncated file.
static int load_device(FileIO& io, void* dst, size_t bytes, cudaStream_t s) {
  unsigned char* p = static_cast<unsigned char*>(dst);
  for (size_t off = 0; off < bytes; off += kStagingBytes) {
    const size_t n = std::min(kStagingBytes, bytes - off);
    if (!io.get(io.staging, n)) return ferror(io.f) ? RGG_ERR_IO : RGG_ERR_INVALID;
    RGG_CK(cudaMemcpyAsync(p + off, io.staging, n, cudaMemcpyHostToDevice, s));
    RGG_CK(cudaStreamSynchronize(s));
  }
  return RGG_OK;
}

int rgg_save(rgg_roadmap_t r, const char* path, void* stream) {
  TraceRange trace_("rgg_save");
  if (!r || !path) return RGG_ERR_INVALID;
  if (!r->has_edges || !r->pending.empty() || r->geometry != RGG_GEOMETRY_SPHERES)
    return RGG_ERR_STATE;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RGG_CK(cudaStreamSynchronize(s));
  const EdgeState& es = r->es;
  FileIO io;
  RGG_CK(cudaMallocHost(reinterpret_cast<void**>(&io.staging), kStagingBytes));
  io.f = std::fopen(path, "wb");
  if (!io.f) return RGG_ERR_IO;
  SaveHeader h{};
  std::memcpy(h.magic, kSaveMagic, 8);
  h.version = 2;
  h.L = r->L;
  h.K = r->K;
  h.M = r->M;
  h.Wm = r->Wm;
  h.margin = r->margin;
  h.flags = (es.regular ? 1u : 0u) | (es.joints ? 2u : 0u);
  h.N = es.N;
  h.S = es.S_tot;
  h.n_inner = es.n_inner;
  h.n_outer = es.n_outer;
  if (!io.put(&h, sizeof(h)) || !io.put(es.h_soff.data(), (es.N + 1) * sizeof(uint64_t)))
    return RGG_ERR_IO;
  int rc = RGG_OK;
  for (int p = 0; p < (es.joints ? 3 : 4) && rc == RGG_OK; ++p)
    rc = save_device(io, es.d_inner + p * es.in_stride, es.n_inner * 4, s);
  if (rc == RGG_OK && es.joints)
    rc = save_device(io, r->d_changed + kBoxesPerPass * kBoxRecFloats,
                     kLinkRadiiFloats * sizeof(float), s);
  for (int p = 0; p < 4 && rc == RGG_OK; ++p)
    rc = save_device(io, es.d_outer + p * es.out_stride, es.n_outer * 4, s);
  const size_t set_bytes = es.N * r->Wm * sizeof(uint32_t);
  if (rc == RGG_OK) rc = save_device(io, es.d_red, set_bytes, s);
  if (rc == RGG_OK) rc = save_device(io, es.d_touch, set_bytes, s);
  if (rc == RGG_OK) rc = save_device(io, es.d_counts, es.N * sizeof(uint32_t), s);
  if (rc == RGG_OK) rc = save_device(io, es.d_labels, es.N, s);
  if (rc == RGG_OK) rc = save_device(io, r->d_table, (size_t)r->M * 16 * sizeof(float), s);
  if (rc == RGG_OK && !io.put(r->present.data(), r->M)) rc = RGG_ERR_IO;
  if (rc != RGG_OK) return rc;
  const uint64_t digest = io.hash.digest();
  if (std::fwrite(&digest, sizeof(digest), 1, io.f) != 1) return RGG_ERR_IO;
  const int closed = std::fclose(io.f);
  io.f = nullptr;
  return closed == 0 ? RGG_OK : RGG_ERR_IO;
}

int rgg_load(rgg_roadmap_t r, const char* path, void* stream) {
  TraceRange trace_("rgg_load");
  if (!r || !path) return RGG_ERR_INVALID;
  if (r->geometry != RGG_GEOMETRY_SPHERES) return RGG_ERR_STATE;
  DeviceGuard g(r->device);
  if (!g.ok) return RGG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  FileIO io;
  io.f = std::fopen(path, "rb");
  if (!io.f) return RGG_ERR_IO;
  SaveHeader h{};
  if (!io.get(&h, sizeof(h))) return ferror(io.f) ? RGG_ERR_IO : RGG_ERR_INVALID;
  const bool joints = (h.flags & 2u) != 0;
  if (std::memcmp(h.magic, kSaveMagic, 8) != 0 || (h.version != 1 && h.version != 2) ||
      (h.version == 1 && joints) || h.L != r->L || h.K != r->K || h.M != r->M || h.Wm != r->Wm ||
      h.N >= 0xffffffffull || h.S < 2 * h.N ||
      h.n_inner != (joints ? 1ull : (uint64_t)h.K) * h.L * h.S ||
      h.n_outer != (uint64_t)h.L * (h.S - h.N))
    return RGG_ERR_INVALID;
  std::vector<uint64_t> soff(h.N + 1);
  if (!io.get(soff.data(), soff.size() * sizeof(uint64_t)))
    return ferror(io.f) ? RGG_ERR_IO : RGG_ERR_INVALID;
  if (!valid_soff(soff.data(), h.N, r->L) || soff[h.N] != h.S) return RGG_ERR_INVALID;
  RGG_CK(cudaMallocHost(reinterpret_cast<void**>(&io.staging), kStagingBytes));
  EdgeState es;
  ShapeRestore shape(r);
  default_shape(r, joints);
  int rc = alloc_edges(r, &es, h.N, std::move(soff), s, joints);
  if (rc != RGG_OK) return rc;
  float link_r[kLinkRadiiFloats] = {};
  float* d_table = nullptr;
  cudaError_t e = dalloc(&d_table, (size_t)r->M * 16);
  if (e != cudaSuccess) {
    es.release();
    return cuda_status(e);
  }
  std::vector<uint8_t> present(r->M);
  for (int p = 0; p < (joints ? 3 : 4) && rc == RGG_OK; ++p)
    rc = load_device(io, es.d_inner + p * es.in_stride, es.n_inner * 4, s);
  if (rc == RGG_OK && joints && !io.get(link_r, sizeof(link_r)))
    rc = ferror(io.f) ? RGG_ERR_IO : RGG_ERR_INVALID;
  for (int p = 0; p < 4 && rc == RGG_OK; ++p)
    rc = load_device(io, es.d_outer + p * es.out_stride, es.n_outer * 4, s);
  const size_t set_bytes = es.N * r->Wm * sizeof(uint32_t);
  if (rc == RGG_OK) rc = load_device(io, es.d_red, set_bytes, s);
  if (rc == RGG_OK) rc = load_device(io, es.d_touch, set_bytes, s);
  if (rc == RGG_OK) rc = load_device(io, es.d_counts, es.N * sizeof(uint32_t), s);
  if (rc == RGG_OK) rc = load_device(io, es.d_labels, es.N, s);
  if (rc == RGG_OK) rc = load_device(io, d_table, (size_t)r->M * 16 * sizeof(float), s);
  if (rc == RGG_OK && !io.get(present.data(), r->M))
    rc = ferror(io.f) ? RGG_ERR_IO : RGG_ERR_INVALID;
  uint64_t stored = 0;
  if (rc == RGG_OK && std::fread(&stored, sizeof(stored), 1, io.f) != 1) rc = RGG_ERR_INVALID;
  if (rc == RGG_OK && stored != io.hash.digest()) rc = RGG_ERR_INVALID;
  if (rc != RGG_OK) {
    es.release();
    device_free(d_table);
    return rc;
  }
  // the file checks out: swap in the edges, the state and the boxes
  es.regular = (h.flags & 1u) != 0;
  e = cudaMemcpyAsync(r->d_table, d_table, (size_t)r->M * 16 * sizeof(float),
                      cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && joints)
    e = cudaMemcpyAsync(r->d_changed + kBoxesPerPass * kBoxRecFloats, link_r, sizeof(link_r),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  device_free(d_table);
  if (e != cudaSuccess) {
    es.release();
    return cuda_status(e);
  }
  rc = compute_rounds(r, &es, s);
  if (rc != RGG_OK) {
    es.release();
    return rc;
  }
  for (uint32_t b = 0; b < r->M; ++b) r->present[b] = present[b] ? 1 : 0;
  shape.keep = true;
  r->es.release();
  r->es = std::move(es);
  r->has_edges = true;
  r->has_robot = false;
  ++r->gen;
  clear_pending(r);
  std::fill(r->req_state.begin(), r->req_state.end(), 0);
  return RGG_OK;
}

}  // extern "C"
