// Bounds-checked builds (check.cuh): the record reader over every
// instrumented kernel file and a self-test of the check itself.
//
// Each instrumented translation unit keeps its own device record and defines
// a reader (AIRGA_CHECK_READER); airga_debug_checked() reads and clears all
// of them.  In normal builds both entry points return AIRGA_E_UNSUPPORTED.
#include "airga_internal.cuh"
#include "check.cuh"

#ifdef AIRGA_CHECKED
namespace airga {
int check_read_pcg_pair(unsigned long long *out);
int check_read_pcg_kernel(unsigned long long *out);
int check_read_pcg_csr(unsigned long long *out);
int check_read_csr_kernels(unsigned long long *out);
int check_read_spai_csr(unsigned long long *out);
int check_read_spai_kernels(unsigned long long *out);
int check_read_mixed(unsigned long long *out);
int check_read_checked(unsigned long long *out);

namespace {
// One thread tests `index` against [0, bound) with the kernels' check; no
// memory at `index` is touched, so any value is safe.
__global__ void check_selftest_kernel(long long index, long long bound, int site) {
    if (threadIdx.x == 0 && blockIdx.x == 0) (void)AIRGA_CK(index, 0, bound, site);
}
}  // namespace
}  // namespace airga

AIRGA_CHECK_READER(checked)
#endif

using namespace airga;

extern "C" int airga_debug_checked(int64_t *violations, int32_t *first_site,
                                   int64_t *first_index) {
    if (!violations) return fail(AIRGA_E_INVALID_ARG, "violations is NULL");
#ifdef AIRGA_CHECKED
    AIRGA_CUDA(cudaDeviceSynchronize());
    int (*const readers[])(unsigned long long *) = {
        check_read_pcg_pair,  check_read_pcg_kernel,   check_read_pcg_csr,
        check_read_csr_kernels, check_read_spai_csr,   check_read_spai_kernels,
        check_read_mixed,     check_read_checked};
    unsigned long long total = 0, site = 0, index = 0;
    for (auto rd : readers) {
        unsigned long long rec[3] = {0ull, 0ull, 0ull};
        if (rd(rec)) return fail(AIRGA_E_CUDA, "reading the bounds-check record failed");
        if (rec[0] && !total) {
            site = rec[1];
            index = rec[2];
        }
        total += rec[0];
    }
    *violations = (int64_t)total;
    if (first_site) *first_site = (int32_t)site;
    if (first_index) *first_index = (int64_t)index;
    return AIRGA_OK;
#else
    (void)first_site;
    (void)first_index;
    *violations = 0;
    return fail(AIRGA_E_UNSUPPORTED, "the library was built without bounds checks");
#endif
}

extern "C" int airga_debug_check_selftest(int64_t index, int64_t bound, int32_t site,
                                          void *stream) {
    if (bound < 0) return fail(AIRGA_E_INVALID_ARG, "bound must be >= 0");
#ifdef AIRGA_CHECKED
    check_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>((long long)index,
                                                             (long long)bound, (int)site);
    AIRGA_CUDA(cudaGetLastError());
    return AIRGA_OK;
#else
    (void)index;
    (void)site;
    (void)stream;
    return fail(AIRGA_E_UNSUPPORTED, "the library was built without bounds checks");
#endif
}
