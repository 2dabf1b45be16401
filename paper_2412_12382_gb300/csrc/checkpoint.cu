// Picker checkpoints as files (tec_picker_file_write / _read, tec_picker_save /
// _load).  Host code only; the format is fixed byte by byte so a file written
// on one machine loads on any other:
//
//   offset  size           field
//   0       8              magic "TECPICK1"
//   8       4              format version (1)
//   12      4              inputs  (TEC_PICKER_INPUTS)
//   16      4              hidden  (TEC_PICKER_HIDDEN)
//   20      4              parameter count (TEC_PICKER_PARAMS)
//   24      8              Adam step count (signed)
//   32      4              meta length L (bytes of UTF-8 text, no terminator)
//   36      L              meta text
//   36+L    4 P            parameters, IEEE binary32
//   ...     4 P            Adam first moments
//   ...     4 P            Adam second moments
//   end-8   8              FNV-1a 64-bit hash of every byte before it
// All integers and floats are little-endian.
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "tec_internal.cuh"

namespace tec {
namespace {

constexpr char MAGIC[8] = {'T', 'E', 'C', 'P', 'I', 'C', 'K', '1'};
constexpr uint32_t VERSION = 1;
constexpr uint32_t META_MAX = 1u << 20;
constexpr size_t HEADER = 36;

// FNV-1a, 64-bit (Fowler, Noll and Vo): offset basis and prime of the
// published definition.
uint64_t fnv1a64(const unsigned char *p, size_t len) {
    uint64_t h = 14695981039346656037ull;
    for (size_t i = 0; i < len; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

void put_u32(std::vector<unsigned char> &b, uint32_t v) {
    for (int i = 0; i < 4; ++i) b.push_back((unsigned char)(v >> (8 * i)));
}
void put_u64(std::vector<unsigned char> &b, uint64_t v) {
    for (int i = 0; i < 8; ++i) b.push_back((unsigned char)(v >> (8 * i)));
}
uint32_t get_u32(const unsigned char *p) {
    uint32_t v = 0;
    for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i);
    return v;
}
uint64_t get_u64(const unsigned char *p) {
    uint64_t v = 0;
    for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i);
    return v;
}
void put_floats(std::vector<unsigned char> &b, const float *x) {
    for (int i = 0; i < TEC_PICKER_PARAMS; ++i) {
        uint32_t bits;
        std::memcpy(&bits, &x[i], 4);
        put_u32(b, bits);
    }
}
void get_floats(const unsigned char *p, float *x) {
    for (int i = 0; i < TEC_PICKER_PARAMS; ++i) {
        const uint32_t bits = get_u32(p + 4 * (size_t)i);
        std::memcpy(&x[i], &bits, 4);
    }
}

// Reads and checks a whole file; on success `buf` holds its bytes and
// *meta_len the meta length.
tec_status read_file(const char *path, std::vector<unsigned char> &buf, uint32_t *meta_len) {
    FILE *f = std::fopen(path, "rb");
    if (!f) return set_error(TEC_EIO, "cannot open %s for reading", path);
    unsigned char chunk[1 << 16];
    size_t got;
    while ((got = std::fread(chunk, 1, sizeof(chunk), f)) > 0) {
        buf.insert(buf.end(), chunk, chunk + got);
        if (buf.size() > (size_t)META_MAX + HEADER + 12 * (size_t)TEC_PICKER_PARAMS + 8) {
            std::fclose(f);
            return set_error(TEC_EIO, "%s is larger than any picker checkpoint", path);
        }
    }
    const bool err = std::ferror(f) != 0;
    std::fclose(f);
    if (err) return set_error(TEC_EIO, "read error on %s", path);
    if (buf.size() < HEADER + 8 || std::memcmp(buf.data(), MAGIC, 8) != 0)
        return set_error(TEC_EIO, "%s is not a picker checkpoint", path);
    if (get_u32(&buf[8]) != VERSION) return set_error(TEC_EIO, "%s: unknown format version %u", path, get_u32(&buf[8]));
    if (get_u32(&buf[12]) != TEC_PICKER_INPUTS || get_u32(&buf[16]) != TEC_PICKER_HIDDEN ||
        get_u32(&buf[20]) != TEC_PICKER_PARAMS)
        return set_error(TEC_EIO, "%s holds another network shape", path);
    const uint32_t L = get_u32(&buf[32]);
    if (L > META_MAX || buf.size() != HEADER + L + 12 * (size_t)TEC_PICKER_PARAMS + 8)
        return set_error(TEC_EIO, "%s has the wrong size", path);
    if (fnv1a64(buf.data(), buf.size() - 8) != get_u64(&buf[buf.size() - 8]))
        return set_error(TEC_EIO, "%s fails its checksum", path);
    *meta_len = L;
    return TEC_OK;
}

}  // namespace
}  // namespace tec

using namespace tec;

extern "C" {

tec_status tec_picker_file_write(const char *path, const float *params, const float *adam_m, const float *adam_v,
                                 int64_t step, const char *meta) {
    clear_error();
    if (!path || !params) return set_error(TEC_EINVAL, "NULL argument");
    const size_t L = meta ? std::strlen(meta) : 0;
    if (L > META_MAX) return set_error(TEC_EINVAL, "meta text longer than %u bytes", META_MAX);
    std::vector<unsigned char> b;
    try {
        b.reserve(HEADER + L + 12 * (size_t)TEC_PICKER_PARAMS + 8);
    } catch (...) {
        return set_error(TEC_ENOMEM, "host allocation failed");
    }
    b.insert(b.end(), MAGIC, MAGIC + 8);
    put_u32(b, VERSION);
    put_u32(b, TEC_PICKER_INPUTS);
    put_u32(b, TEC_PICKER_HIDDEN);
    put_u32(b, TEC_PICKER_PARAMS);
    put_u64(b, (uint64_t)step);
    put_u32(b, (uint32_t)L);
    b.insert(b.end(), meta, meta + L);
    std::vector<float> zeros;
    if (!adam_m || !adam_v) zeros.assign(TEC_PICKER_PARAMS, 0.f);
    put_floats(b, params);
    put_floats(b, adam_m ? adam_m : zeros.data());
    put_floats(b, adam_v ? adam_v : zeros.data());
    put_u64(b, fnv1a64(b.data(), b.size()));
    FILE *f = std::fopen(path, "wb");
    if (!f) return set_error(TEC_EIO, "cannot open %s for writing", path);
    const bool ok = std::fwrite(b.data(), 1, b.size(), f) == b.size();
    const bool closed = std::fclose(f) == 0;
    if (!ok || !closed) return set_error(TEC_EIO, "write error on %s", path);
    return TEC_OK;
}

tec_status tec_picker_file_read(const char *path, float *params, float *adam_m, float *adam_v, int64_t *step,
                                char *meta, size_t meta_cap, size_t *meta_len) {
    clear_error();
    if (!path) return set_error(TEC_EINVAL, "path is NULL");
    std::vector<unsigned char> buf;
    uint32_t L = 0;
    try {
        TEC_TRY(read_file(path, buf, &L));
    } catch (...) {
        return set_error(TEC_ENOMEM, "host allocation failed");
    }
    const unsigned char *p = buf.data() + HEADER + L;
    if (params) get_floats(p, params);
    if (adam_m) get_floats(p + 4 * (size_t)TEC_PICKER_PARAMS, adam_m);
    if (adam_v) get_floats(p + 8 * (size_t)TEC_PICKER_PARAMS, adam_v);
    if (step) *step = (int64_t)get_u64(&buf[24]);
    if (meta_len) *meta_len = L;
    if (meta && meta_cap > 0) {
        const size_t c = L < meta_cap - 1 ? L : meta_cap - 1;
        std::memcpy(meta, buf.data() + HEADER, c);
        meta[c] = '\0';
    }
    return TEC_OK;
}

tec_status tec_picker_save(tec_picker *p, const char *path, const char *meta) {
    clear_error();
    if (!p || !path) return set_error(TEC_EINVAL, "NULL argument");
    std::vector<float> h;
    try {
        h.resize(3 * (size_t)TEC_PICKER_PARAMS);
    } catch (...) {
        return set_error(TEC_ENOMEM, "host allocation failed");
    }
    int64_t step = 0;
    TEC_TRY(tec_picker_get_params(p, h.data(), h.data() + TEC_PICKER_PARAMS, h.data() + 2 * TEC_PICKER_PARAMS,
                                  &step));
    return tec_picker_file_write(path, h.data(), h.data() + TEC_PICKER_PARAMS, h.data() + 2 * TEC_PICKER_PARAMS,
                                 step, meta);
}

tec_status tec_picker_load(const char *path, void *stream, tec_picker **out) {
    clear_error();
    if (!path || !out) return set_error(TEC_EINVAL, "NULL argument");
    *out = nullptr;
    std::vector<float> h;
    try {
        h.resize(3 * (size_t)TEC_PICKER_PARAMS);
    } catch (...) {
        return set_error(TEC_ENOMEM, "host allocation failed");
    }
    int64_t step = 0;
    TEC_TRY(tec_picker_file_read(path, h.data(), h.data() + TEC_PICKER_PARAMS, h.data() + 2 * TEC_PICKER_PARAMS,
                                 &step, nullptr, 0, nullptr));
    tec_picker *p = nullptr;
    TEC_TRY(tec_picker_create(h.data(), stream, &p));
    const tec_status s = tec_picker_set_params(p, h.data(), h.data() + TEC_PICKER_PARAMS,
                                               h.data() + 2 * TEC_PICKER_PARAMS, step);
    if (s != TEC_OK) {
        tec_picker_free(p);
        return set_error(s, "setting the parameters read from %s failed", path);
    }
    *out = p;
    return TEC_OK;
}

}  // extern "C"
