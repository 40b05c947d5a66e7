// Serialisation of packed handles: a pre-packed weight (Sec. 4.1 packs A once
// for inference, and the pack is reused by every SpMM) is written to a byte
// image and restored in another process without re-running the pack.
//
// Image (little-endian, every field naturally aligned):
//   Header          fixed-size fields (magic, format version, sizes, array
//                   offsets inside the device allocation, vector lengths)
//   host vectors    the handle's host-side bookkeeping (segment prefix sums,
//                   dense-tile order and densities, panel offsets)
//   device blob     the handle's single device allocation, byte for byte
//   checksum        FNV-1a (64 bit) of everything before it
// Device arrays are stored as offsets from the allocation's base, so a
// restored handle rebuilds its pointers from its own new allocation.
#include <cstring>
#include <new>
#include <vector>

#include "handle.hpp"

namespace rosko {
namespace {

constexpr uint64_t kImageMagic = 0x31504b4f4b534f52ull;  // "ROSKOKP1"
constexpr uint32_t kImageVersion = 1;
constexpr int kNumPtrs = 20;

struct Header {
  uint64_t magic;
  uint32_t version, header_bytes;
  int32_t dt, m_r;
  int64_t M, K, P, nnz, n_cols, touched_k, gu_total, n_tiles, n_copy, Kpad;
  uint64_t base_bytes;
  int64_t ptr_off[kNumPtrs];   // -1: null
  int32_t seg_records[2];
  int64_t n_prefix[2], n_split[2];
  int64_t n_tile_order, n_panel_order, n_tile_density, n_tile_panels, n_panel_nnz;
};

uint64_t fnv1a(const unsigned char* p, size_t n, uint64_t h = 1469598103934665603ull) {
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

// The device pointers of a handle, in image order.
void** ptr_slots(rosko_packed_s* h, void** slots[kNumPtrs]) {
  int i = 0;
  slots[i++] = reinterpret_cast<void**>(&h->panel_col);
  slots[i++] = reinterpret_cast<void**>(&h->colrec);
  slots[i++] = &h->nz;
  slots[i++] = reinterpret_cast<void**>(&h->row_scale);
  slots[i++] = reinterpret_cast<void**>(&h->rowptr);
  slots[i++] = &h->rnz;
  slots[i++] = reinterpret_cast<void**>(&h->gu_start);
  slots[i++] = reinterpret_cast<void**>(&h->gu_k);
  slots[i++] = &h->gnz;
  slots[i++] = reinterpret_cast<void**>(&h->feat_dev);
  slots[i++] = reinterpret_cast<void**>(&h->panel_nnz_dev);
  slots[i++] = &h->dense_A;
  slots[i++] = reinterpret_cast<void**>(&h->tile_order_dev);
  slots[i++] = reinterpret_cast<void**>(&h->panel_order_dev);
  slots[i++] = reinterpret_cast<void**>(&h->segs[0].nat);
  slots[i++] = reinterpret_cast<void**>(&h->segs[0].ord);
  slots[i++] = reinterpret_cast<void**>(&h->segs[1].nat);
  slots[i++] = reinterpret_cast<void**>(&h->segs[1].ord);
  slots[i++] = reinterpret_cast<void**>(&h->segs[0].lpt);
  slots[i++] = reinterpret_cast<void**>(&h->segs[1].lpt);
  return slots[0];
}

template <class T>
void put(std::vector<unsigned char>& out, const std::vector<T>& v) {
  const size_t at = out.size();
  out.resize(at + v.size() * sizeof(T));
  if (!v.empty()) std::memcpy(out.data() + at, v.data(), v.size() * sizeof(T));
}

template <class T>
bool get(const unsigned char* buf, size_t size, size_t* at, int64_t n, std::vector<T>* v) {
  if (n < 0 || (uint64_t)n > (size - *at) / sizeof(T)) return false;
  v->resize((size_t)n);
  if (n) std::memcpy(v->data(), buf + *at, (size_t)n * sizeof(T));
  *at += (size_t)n * sizeof(T);
  return true;
}

}  // namespace

rosko_status packed_serialize(const rosko_packed_s* hc, void* buf, int64_t cap, int64_t* bytes) {
  rosko_packed_s* h = const_cast<rosko_packed_s*>(hc);
  Header H;
  std::memset(&H, 0, sizeof(H));
  H.magic = kImageMagic;
  H.version = kImageVersion;
  H.header_bytes = (uint32_t)sizeof(Header);
  H.dt = (int32_t)h->dt;
  H.m_r = h->m_r;
  H.M = h->M;
  H.K = h->K;
  H.P = h->P;
  H.nnz = h->nnz;
  H.n_cols = h->n_cols;
  H.touched_k = h->touched_k;
  H.gu_total = h->gu_total;
  H.n_tiles = h->n_tiles;
  H.n_copy = h->n_copy;
  H.Kpad = h->Kpad;
  H.base_bytes = h->base_bytes;
  void** slots[kNumPtrs];
  ptr_slots(h, slots);
  for (int i = 0; i < kNumPtrs; ++i) {
    const char* p = static_cast<const char*>(*slots[i]);
    H.ptr_off[i] = p ? (int64_t)(p - static_cast<const char*>(h->base)) : -1;
  }
  for (int g = 0; g < 2; ++g) {
    H.seg_records[g] = h->segs[g].records;
    H.n_prefix[g] = (int64_t)h->segs[g].prefix.size();
    H.n_split[g] = (int64_t)h->segs[g].split.size();
  }
  H.n_tile_order = (int64_t)h->tile_order.size();
  H.n_panel_order = (int64_t)h->panel_order_host.size();
  H.n_tile_density = (int64_t)h->tile_density.size();
  H.n_tile_panels = (int64_t)h->tile_panels.size();
  H.n_panel_nnz = (int64_t)h->panel_nnz.size();
  std::vector<unsigned char> img(sizeof(Header));
  std::memcpy(img.data(), &H, sizeof(Header));
  for (int g = 0; g < 2; ++g) {
    put(img, h->segs[g].prefix);
    put(img, h->segs[g].split);
  }
  put(img, h->tile_order);
  put(img, h->panel_order_host);
  put(img, h->tile_density);
  put(img, h->tile_panels);
  put(img, h->panel_nnz);
  const size_t blob = img.size();
  const int64_t total = (int64_t)(blob + h->base_bytes + sizeof(uint64_t));
  *bytes = total;
  if (!buf) return ROSKO_OK;            // size query
  if (cap < total) return ROSKO_ERR_INVALID_ARG;
  unsigned char* out = static_cast<unsigned char*>(buf);
  std::memcpy(out, img.data(), blob);
  // every queued write of the handle (the pack) has finished: rosko_pack
  // synchronises before returning; the copy below is ordered after it
  if (h->base_bytes &&
      cudaMemcpy(out + blob, h->base, h->base_bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ROSKO_ERR_CUDA;
  const uint64_t sum = fnv1a(out, blob + h->base_bytes);
  std::memcpy(out + blob + h->base_bytes, &sum, sizeof(sum));
  return ROSKO_OK;
}

rosko_status packed_deserialize(const void* vbuf, int64_t size, cudaStream_t st,
                                rosko_packed_s** out) {
  *out = nullptr;
  const unsigned char* buf = static_cast<const unsigned char*>(vbuf);
  if (size < (int64_t)(sizeof(Header) + sizeof(uint64_t))) return ROSKO_ERR_INVALID_ARG;
  Header H;
  std::memcpy(&H, buf, sizeof(Header));
  if (H.magic != kImageMagic) return ROSKO_ERR_INVALID_ARG;
  // damage first (any version), then the format version
  uint64_t want = 0;
  std::memcpy(&want, buf + size - sizeof(uint64_t), sizeof(want));
  if (fnv1a(buf, (size_t)size - sizeof(uint64_t)) != want) return ROSKO_ERR_INVALID_ARG;
  if (H.version != kImageVersion || H.header_bytes != sizeof(Header)) return ROSKO_ERR_UNSUPPORTED;
  if (!dtype_valid(H.dt) || (H.m_r != 8 && H.m_r != 16 && H.m_r != 32) || H.M < 0 || H.K < 0 ||
      H.P != (H.M + H.m_r - 1) / H.m_r || H.nnz < 0 || H.base_bytes < 256)
    return ROSKO_ERR_INVALID_ARG;
  rosko_packed_s* h = new (std::nothrow) rosko_packed_s();
  if (!h) return ROSKO_ERR_OOM;
  size_t at = sizeof(Header);
  const size_t body = (size_t)size - sizeof(uint64_t);
  bool ok = true;
  for (int g = 0; g < 2 && ok; ++g) {
    ok = get(buf, body, &at, H.n_prefix[g], &h->segs[g].prefix) &&
         get(buf, body, &at, H.n_split[g], &h->segs[g].split);
    h->segs[g].records = H.seg_records[g];
  }
  ok = ok && get(buf, body, &at, H.n_tile_order, &h->tile_order) &&
       get(buf, body, &at, H.n_panel_order, &h->panel_order_host) &&
       get(buf, body, &at, H.n_tile_density, &h->tile_density) &&
       get(buf, body, &at, H.n_tile_panels, &h->tile_panels) &&
       get(buf, body, &at, H.n_panel_nnz, &h->panel_nnz);
  if (!ok || body - at != H.base_bytes) {
    delete h;
    return ROSKO_ERR_INVALID_ARG;
  }
  for (int i = 0; i < kNumPtrs; ++i)
    if (H.ptr_off[i] < -1 || H.ptr_off[i] >= (int64_t)H.base_bytes) {
      delete h;
      return ROSKO_ERR_INVALID_ARG;
    }
  h->dt = (rosko_dtype)H.dt;
  h->m_r = H.m_r;
  h->M = H.M;
  h->K = H.K;
  h->P = H.P;
  h->nnz = H.nnz;
  h->n_cols = H.n_cols;
  h->touched_k = H.touched_k;
  h->gu_total = H.gu_total;
  h->n_tiles = H.n_tiles;
  h->n_copy = H.n_copy;
  h->Kpad = H.Kpad;
  cudaGetDevice(&h->device);
  if (pool_malloc(&h->base, H.base_bytes, st) != cudaSuccess) {
    delete h;
    return ROSKO_ERR_OOM;
  }
  h->base_bytes = H.base_bytes;
  void** slots[kNumPtrs];
  ptr_slots(h, slots);
  for (int i = 0; i < kNumPtrs; ++i)
    *slots[i] = H.ptr_off[i] < 0 ? nullptr : static_cast<char*>(h->base) + H.ptr_off[i];
  // a pageable source: the copy is complete when the call returns
  if (cudaMemcpyAsync(h->base, buf + at, H.base_bytes, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    pool_free(h->base, st);
    delete h;
    return ROSKO_ERR_CUDA;
  }
  h->magic = kHandleMagic;
  *out = h;
  return ROSKO_OK;
}

}  // namespace rosko
