// Checkpoint file of the training state: weights, Adam moments and step
// counts (Section 4 trains with Adam; the state that a resumed run needs).
// Host code only; hrkan_save / hrkan_load (capi.cu) move the device state.
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/hrkan.h"
#include "internal.h"

namespace {

constexpr char MAGIC[8] = {'H', 'R', 'K', 'A', 'N', 'C', 'K', '1'};
constexpr uint32_t VERSION = 1;

struct Header {
    char magic[8];
    uint32_t version;
    uint32_t n_instances;
    int64_t P;
    int64_t t;
    int64_t t_device;
};
static_assert(sizeof(Header) == 40, "packed header");

int io_fail(const char* what, const char* path) {
    std::string m = std::string("checkpoint: ") + what + " '" + path + "'";
    return hrkan::set_last_error(HRKAN_EIO, m.c_str());
}

bool write_all(FILE* f, const void* p, size_t bytes) { return bytes == 0 || fwrite(p, 1, bytes, f) == bytes; }
bool read_all(FILE* f, void* p, size_t bytes) { return bytes == 0 || fread(p, 1, bytes, f) == bytes; }

}  // namespace

extern "C" {

int hrkan_checkpoint_write(const char* path, int64_t P, int n_instances, int64_t t, int64_t t_device, const float* W,
                           const double* m, const double* v) {
    if (!path || !W || !m || !v || P <= 0 || n_instances <= 0)
        return hrkan::set_last_error(HRKAN_EINVAL, "hrkan_checkpoint_write: null pointer or empty state");
    Header h{};
    std::memcpy(h.magic, MAGIC, 8);
    h.version = VERSION;
    h.n_instances = uint32_t(n_instances);
    h.P = P;
    h.t = t;
    h.t_device = t_device;
    const size_t n = size_t(P) * size_t(n_instances);
    // write a sibling file and rename it over the target: a crash never leaves a torn checkpoint
    const std::string tmp = std::string(path) + ".part";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return io_fail("cannot create", tmp.c_str());
    bool ok = write_all(f, &h, sizeof h) && write_all(f, W, n * sizeof(float)) && write_all(f, m, n * sizeof(double)) &&
              write_all(f, v, n * sizeof(double));
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) {
        std::remove(tmp.c_str());
        return io_fail("cannot write", tmp.c_str());
    }
    if (std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return io_fail("cannot rename onto", path);
    }
    return HRKAN_OK;
}

int hrkan_checkpoint_read(const char* path, int64_t P, int n_instances, int64_t* t, int64_t* t_device, float* W,
                          double* m, double* v) {
    if (!path || !W || !m || !v || P <= 0 || n_instances <= 0)
        return hrkan::set_last_error(HRKAN_EINVAL, "hrkan_checkpoint_read: null pointer or empty state");
    FILE* f = std::fopen(path, "rb");
    if (!f) return io_fail("cannot open", path);
    Header h{};
    if (!read_all(f, &h, sizeof h) || std::memcmp(h.magic, MAGIC, 8) != 0 || h.version != VERSION) {
        std::fclose(f);
        return io_fail("not a version-1 HRKAN checkpoint:", path);
    }
    if (h.P != P || int64_t(h.n_instances) != int64_t(n_instances)) {
        std::fclose(f);
        char buf[200];
        std::snprintf(buf, sizeof buf, "checkpoint holds %u x %lld weights, the network has %d x %lld",
                      h.n_instances, (long long)h.P, n_instances, (long long)P);
        return hrkan::set_last_error(HRKAN_EINVAL, buf);
    }
    const size_t n = size_t(P) * size_t(n_instances);
    const bool ok = read_all(f, W, n * sizeof(float)) && read_all(f, m, n * sizeof(double)) &&
                    read_all(f, v, n * sizeof(double));
    char extra;
    const bool at_end = ok && std::fread(&extra, 1, 1, f) == 0;
    std::fclose(f);
    if (!ok) return io_fail("truncated", path);
    if (!at_end) return io_fail("trailing bytes in", path);
    if (t) *t = h.t;
    if (t_device) *t_device = h.t_device;
    return HRKAN_OK;
}

}  // extern "C"
