// fm_sched.h -- the aligned / contained decomposition as flat work lists.
//
// Sec. 2.2 recurses on the aligned parents of the three operands so that every
// base case multiplies parts that each lie inside one row-major T' x T' tile
// (Prop. and Cor. of Sec. 2.1). Its leaves are exactly the cells of three
// interval partitions of the product's local index space:
//   i (rows of C and A)     cut at the tile-row boundaries of C and of A,
//   j (columns of C and B)  cut at the tile-column boundaries of C and of B,
//   l (inner index)         cut at the tile-column boundaries of A and the
//                           tile-row boundaries of B.
// The scheduler emits them grouped by output tile: one work item per part of
// C inside one C tile (rows and columns cut at C's boundaries), carrying the
// at-most-one cut of A's rows and of B's columns inside it, plus a shared list
// of l-pieces. A work item with its l-pieces and the two cuts is the flat list
// of contiguous tile triples the kernels consume.
#pragma once

#include <stdint.h>

#include <vector>

#include "fm.h"

// Device view of one call: matrix bases and parameters.
struct FmCallDesc {
    uint32_t* C;
    const uint32_t* A;
    const uint32_t* B;
    int32_t lt;   // log2 T' (shared by C, A and B for the decomposed paths)
    int32_t op;   // fm_op
    int32_t lp_begin, lp_count;  // this call's l-pieces in the shared list
};

// One output part: rows x cols of C inside C tile (c_ti, c_tj), starting at
// in-tile (c_r, c_c). Its local row x (0 <= x < rows) reads A tile row a_ti
// at in-tile row a_r + x while x < a_split, then tile row a_ti + 1 at in-tile
// row a_r + x - T'. Its local column y reads B tile column b_tj at in-tile
// column b_c + y while y < b_split, then tile column b_tj + 1.
struct FmWorkItem {
    int32_t call;
    int32_t c_ti, c_tj, c_r, c_c, rows, cols;
    int32_t a_ti, a_r, a_split;
    int32_t b_tj, b_c, b_split;
    int32_t i0, j0;  // local offsets of the part inside the product
    int32_t pad;
};

// One inner-index piece: l in [l0, l0 + len) lies in A tile column a_tj at
// in-tile column a_c.. and in B tile row b_ti at in-tile row b_r..
struct FmLPiece {
    int32_t a_tj, a_c, b_ti, b_r, len, l0;
};

// Validates C <- C op A*B operands (shapes, extents, equal T' when
// same_tile is set, no overlap of C with A or B). FM_OK or a negative status.
int fm_check_product(const fm_sub& C, const fm_sub& A, const fm_sub& B, bool same_tile);

// Appends the work items and l-pieces of one call to the lists.
void fm_decompose_call(const fm_sub& C, const fm_sub& A, const fm_sub& B, int32_t call_index,
                       std::vector<FmWorkItem>& items, std::vector<FmLPiece>& lps,
                       int32_t* lp_begin, int32_t* lp_count);
