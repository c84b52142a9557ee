// Bounds-checked build.  Compiled with -DDH_CHECKED (the library libdigholo_gb300_checked.so), every guarded
// global-memory access of the reconstruction kernels first tests its element offset against the extent of the
// buffer it addresses (and every 16-byte vector access its alignment); a failed test skips the access and
// records itself in the plan's status block instead of touching memory outside the buffer:
//   status[0] |= 4 (DH_STATUS_BOUNDS), status[1] = the first failing site (kSite*), status[2] = its offset
//   (low 32 bits), status[3] = the extent (low 32 bits).
// In the normal build every guard is the constant true and compiles away.  A checked run reports an indexing or
// scratch-carving mistake as a status word and a guard site instead of a device fault.
#pragma once

#include <stdint.h>

namespace dhk {

// Guard sites (reported in status[1]).
enum CheckSite : int {
    kSiteNone = 0,
    kSiteYpassR1 = 1,        // k_ypass / k_ypass_s: box-row store into r1 scratch
    kSiteYpassFrame = 2,     // k_ypass / k_ypass_s: pixel load
    kSiteXpassR1 = 3,        // k_xpass / k_xpass_s: box-row load from r1 scratch
    kSiteXpassG = 4,         // k_xpass / k_xpass_s: x-inverse row store into g scratch
    kSiteXpassWindow = 5,    // k_xpass / k_xpass_s: Fourier-window store
    kSiteYinvG = 6,          // k_yinv / k_yinv_tc: g scratch load
    kSiteYinvField = 7,      // k_yinv / k_yinv_tc: field store
    kSiteYinvCoef = 8,       // k_yinv / k_yinv_tc: coefficient store
    kSiteFusedField = 9,     // fused kernels: field store
    kSiteFusedCoef = 10,     // fused kernels: coefficient store
    kSiteFusedWindow = 11,   // fused kernel, split modes: window store / load
    kSiteCoefTcCopy = 12,    // k_coef_tc: bulk-copy source range
    kSiteCoefTcCoef = 13,    // k_coef_tc: coefficient store
    kSiteScore = 14,         // candidate scoring: superset spectra and candidate rows
    kSiteAvg = 15,           // batch averaging: member windows, partial sums, means
    kSiteBasis = 16,         // output-basis transform: coefficient load / store
    kSiteAlign16 = 17,       // a 16-byte vector access on an address that is not 16-byte aligned
    kSiteProbe = 99          // dh_check_bounds_probe
};

#ifdef DH_CHECKED
constexpr bool kChecked = true;

__device__ __forceinline__ bool check_record(int* status, bool ok, int site, long long off, long long lim) {
    if (!ok && status) {
        atomicOr(status, 4);
        if (atomicCAS(status + 1, 0, site) == 0) {
            atomicExch(status + 2, (int)off);
            atomicExch(status + 3, (int)lim);
        }
    }
    return ok;
}

// true when 0 <= off < lim (else recorded at site)
#define DH_IN(status, off, lim, site)                                                                           \
    ::dhk::check_record((status), (unsigned long long)(long long)(off) < (unsigned long long)(long long)(lim), \
                        (site), (long long)(off), (long long)(lim))
// true when the address is 16-byte aligned (else recorded at site kSiteAlign16)
#define DH_ALIGNED16(status, ptr) \
    ::dhk::check_record((status), ((uintptr_t)(ptr) & 15) == 0, ::dhk::kSiteAlign16, (long long)((uintptr_t)(ptr) & 15), 16)
#else
constexpr bool kChecked = false;
#define DH_IN(status, off, lim, site) true
#define DH_ALIGNED16(status, ptr) true
#endif

}  // namespace dhk
