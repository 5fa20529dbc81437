// checks.h -- bounds predicates of the checked mode (options.checked = 1).
//
// Plain inline functions, callable from host and device code, so that the
// host test suite can exercise them without a GPU.  Each names the site whose
// index it guards; a failed check skips the access and records the site in the
// context's device status word (tsp_sync reports it).
#ifndef TSP_CHECKS_H
#define TSP_CHECKS_H

#include <stdint.h>

#if defined(__CUDACC__)
#define TSP_HD __host__ __device__ __forceinline__
#else
#define TSP_HD inline
#endif

namespace tsp {

// Sites, in the order of the pipeline steps (the code tsp_sync reports).
enum CheckSite : uint32_t {
    kSiteNone = 0,
    kSiteScatterTile = 1,     // a2 emit: tile index of a (record, tile) item
    kSiteScatterSlot = 2,     // a2 emit: slot past the end of the tile's list
    kSiteTileRange = 3,       // a3 sort: tile offsets not ascending or past the pair buffer
    kSiteRefPixel = 4,        // reference gather: moment-origin pixel outside the image
    kSiteListEntry = 5,       // a5 raster / render: list entry's Gaussian index past the view's count
    kSiteCount = 6
};

// index < size
TSP_HD bool index_ok(uint64_t index, uint64_t size) { return index < size; }

// [begin, end) is a valid range of a buffer of `size` elements
TSP_HD bool range_ok(uint64_t begin, uint64_t end, uint64_t size) { return begin <= end && end <= size; }

// the slot `fill` of a tile's list [begin, end) stays inside the list
TSP_HD bool slot_ok(uint64_t begin, uint64_t fill, uint64_t end) { return fill < end - begin && begin <= end; }

// pixel index inside a W x H image
TSP_HD bool pixel_ok(uint64_t pix, uint32_t W, uint32_t H) { return pix < (uint64_t)W * (uint64_t)H; }

inline const char* check_site_name(uint32_t site)
{
    switch (site) {
    case kSiteScatterTile: return "emit: tile index of an item";
    case kSiteScatterSlot: return "emit: slot past the end of a tile list";
    case kSiteTileRange: return "tile sort: tile range";
    case kSiteRefPixel: return "reference gather: origin pixel";
    case kSiteListEntry: return "raster: list entry's Gaussian index";
    default: return "unknown site";
    }
}

}  // namespace tsp

#endif
