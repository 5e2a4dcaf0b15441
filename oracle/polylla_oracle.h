/*
 * CPU oracle of the terminal-edge-region polygonal mesher (test infrastructure).
 * See polylla_oracle.c for the layout, the paper passages each routine follows and
 * the readings it fixes.  This header belongs to the oracle alone.
 */
#ifndef POLYLLA_ORACLE_H
#define POLYLLA_ORACLE_H
#include <stdint.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG (-1)
#define ORACLE_ERR_NOT_DISK (-2) /* a region boundary is not one cycle, or a bad tip */
#define ORACLE_ERR_OOM (-3)
#define ORACLE_ERR_CAPACITY (-4)

#ifdef __cplusplus
extern "C" {
#endif

int oracle_label_max(const int64_t* xy, const int32_t* tri, const int32_t* twin, int64_t m,
                     uint8_t* max_edge);
int oracle_label_seed(const int32_t* twin, int64_t m, const uint8_t* max_edge, uint8_t* seed,
                      uint8_t* terminal);
int oracle_label_frontier(const int32_t* twin, int64_t m, const uint8_t* max_edge,
                          uint8_t* frontier);
int64_t oracle_seed_list(const uint8_t* seed, int64_t m, int32_t* seeds);
int64_t oracle_lepp(const int32_t* twin, int64_t m, const uint8_t* max_edge, int32_t* region,
                    int32_t* depth);
int oracle_trivertex(const int32_t* tri, int64_t m, int64_t n, int64_t* tv);
int64_t oracle_traverse(const int32_t* tri, const int32_t* twin, int64_t m, const uint8_t* frontier,
                        const int32_t* seeds, int64_t ns, int64_t* off, int32_t* vtx,
                        int64_t cap_vtx);
int64_t oracle_repair(int64_t n, const int32_t* tri, const int32_t* twin, int64_t m,
                      uint8_t* frontier, const int64_t* off_in, const int32_t* vtx_in,
                      int64_t np_in, int64_t* off_out, int32_t* vtx_out, int64_t cap_poly,
                      int64_t cap_vtx, int64_t* np_out, int64_t* stats);
int64_t oracle_run(const int64_t* xy, int64_t n, const int32_t* tri, const int32_t* twin,
                   int64_t m, uint8_t* max_edge, uint8_t* frontier, int64_t* off, int32_t* vtx,
                   int64_t* np_out, int64_t* stats);

#ifdef __cplusplus
}
#endif
#endif
