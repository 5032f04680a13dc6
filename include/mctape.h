/* mctape.h -- expected-backward automatic differentiation of a whole
 * Monte-Carlo program on the GPU (arXiv 1901.04200, Appendix, after Fries).
 *
 * A program is a list of operations x_m = f_m(x_a, x_b) in topological order
 * (every argument precedes its node).  Values are random variables over the
 * Monte-Carlo paths: a node is deterministic (the same on every path: model
 * parameters, constants, expectations and functions of these) or per-path.
 * One operation is the expectation operator E: its value is the mean of its
 * argument over the evaluated paths.  The objective is a deterministic node.
 *
 * The backward sweep follows the Appendix's rule: starting from D_N = 1 at
 * the objective and walking the list from last to first, an ordinary node m
 * adds D_m * d f_m / d x_j to the adjoint of each argument j, and an
 * expectation node m adds E(D_m) to the adjoint of its argument; the
 * derivative of the objective with respect to parameter k is E(D) of the
 * parameter's node.  Unlike the two-step algorithm of mcaad.h, the program
 * may use an expectation anywhere (inside a path's computation, inside
 * another expectation), and the whole program is differentiated through.
 *
 * GPU execution: the host cuts the program into stages at the first use of
 * each expectation's value.  Per stage, one thread evaluates the
 * deterministic nodes, one GPU thread per path interprets the per-path nodes
 * (values FP64 or FP32, structure of arrays [node][path] in HBM where needed
 * later),
 * and fixed-order block sums then a fixed-order
 * sum over blocks give the stage's expectations.  The backward sweep runs
 * the stages in reverse: per-path adjoints in a second [node][path] array;
 * adjoints of deterministic nodes are means over paths (warp sums, per-warp
 * FP64 accumulators, fixed-order sums over blocks), so results are bitwise
 * reproducible for a given problem.  Normals are those of mcaad.h: normal j
 * of global path p is Philox-4x32-10 block (counter j>>2, path p, key seed),
 * Box-Muller pair (j&3)>>1, member j&1.
 *
 * Status codes and stream conventions are those of mcaad.h.
 */
#ifndef MCTAPE_H
#define MCTAPE_H

#include <stddef.h>
#include <stdint.h>

#include "mcaad.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Operations.  a, b: argument node indices (-1 if unused); c: the constant.
 * Partial derivatives (the kink conventions of mcaad.h):
 *   MC_OP_PARAM   theta[(int)c]                     (deterministic)
 *   MC_OP_CONST   c                                 (deterministic)
 *   MC_OP_NORMAL  normal (int)c of the path         (per path)
 *   MC_OP_ADD a+b, MC_OP_SUB a-b, MC_OP_MUL a*b, MC_OP_DIV a/b
 *   MC_OP_ADDC a+c, MC_OP_MULC a*c, MC_OP_NEG -a
 *   MC_OP_EXP, MC_OP_LOG
 *   MC_OP_SQRT    derivative 1/(2 sqrt a) for a > 0, 0 at a <= 0
 *   MC_OP_RELU    max(a, 0), derivative 1{a > 0}
 *   MC_OP_ABS     |a|, derivative sign(a) (0 at 0)
 *   MC_OP_EXPECT  E(a): the mean over the evaluated paths (deterministic) */
typedef enum {
    MC_OP_PARAM = 0,
    MC_OP_CONST = 1,
    MC_OP_NORMAL = 2,
    MC_OP_ADD = 3,
    MC_OP_SUB = 4,
    MC_OP_MUL = 5,
    MC_OP_DIV = 6,
    MC_OP_ADDC = 7,
    MC_OP_MULC = 8,
    MC_OP_NEG = 9,
    MC_OP_EXP = 10,
    MC_OP_LOG = 11,
    MC_OP_SQRT = 12,
    MC_OP_RELU = 13,
    MC_OP_ABS = 14,
    MC_OP_EXPECT = 15,
    MC_N_OPS = 16
} mc_tape_op;

typedef struct {
    int32_t op;   /* mc_tape_op */
    int32_t a, b; /* argument nodes, < this node's index; -1 if the op takes fewer */
    double c;     /* PARAM: parameter index; CONST, ADDC, MULC: the constant; NORMAL: normal index */
} mc_tape_node;

/* Plan facts of a program, computed on the host (no GPU needed; the stages are
 * cut where an expectation's value is first used, Appendix): checks the
 * program (MC_ERR_INVALID_ARG for an argument index out of range or not
 * preceding its node, an unknown op, a parameter index outside [0,
 * n_params), a negative normal index, an objective that is not
 * deterministic; MC_ERR_UNSUPPORTED above the limits: 2^24 nodes, 2048
 * expectations per stage, 2048 distinct deterministic arguments of one
 * stage's per-path nodes).  Any output pointer may be NULL.
 *   n_stages       stages (expectation boundaries + 1)
 *   n_path_nodes   per-path nodes (rows of the value and adjoint tapes)
 *   workspace      device bytes a context needs for max_paths paths
 *   hbm_bytes      HBM bytes per path that one mc_tape_value_and_grad moves:
 *                  a per-thread shared-memory window holds the last 32
 *                  per-path values (forward) and adjoints (backward) of a
 *                  stage, so only values a far or later-stage user, an
 *                  expectation or a backward partial needs go to the tape */
mc_status mc_tape_plan(const mc_tape_node *nodes, int32_t n_nodes, int32_t objective, int32_t n_params,
                       int32_t precision, uint64_t max_paths, int32_t *n_stages, int32_t *n_path_nodes,
                       size_t *workspace, size_t *hbm_bytes);

typedef struct mc_tape mc_tape;

/* Copy the program to `device` and allocate the tapes for up to max_paths
 * paths (workspace: caller-owned device buffer of mc_tape_plan's bytes,
 * 256-byte aligned, or NULL to let the context allocate).  precision
 * (mc_precision) is that of the per-path values, adjoints and normals:
 * MC_FP64, or MC_FP32 with FP64 kept for the deterministic nodes, the
 * expectations and every sum over paths.  Synchronous. */
mc_status mc_tape_create(int device, const mc_tape_node *nodes, int32_t n_nodes, int32_t objective,
                         int32_t n_params, int32_t precision, uint64_t max_paths, void *workspace,
                         size_t workspace_bytes, mc_tape **out);
void mc_tape_destroy(mc_tape *t);
const char *mc_tape_last_error(const mc_tape *t);

/* The objective and its gradient over global paths [path0, path0 + n_paths)
 * of `seed`: the forward stages, then the backward sweep by the Appendix's
 * rule (expected backward AD after Fries), as described at the top of this
 * file.  theta: FP64 device [n_params]; value_out: FP64 device [1];
 * grad_out: FP64 device [n_params].  Stream-ordered on `stream`. */
mc_status mc_tape_value_and_grad(mc_tape *t, const double *theta, uint64_t seed, uint64_t path0,
                                 uint64_t n_paths, double *value_out, double *grad_out, void *stream);

/* Compile the program (the GPU analogue of a tape compiler): each stage's
 * per-path nodes are cut into segments of seg_nodes consecutive nodes (0: 384)
 * and every segment becomes a straight-line forward kernel (values in
 * registers) and a straight-line backward kernel (adjoints in registers),
 * compiled at run time for sm_103a by NVRTC on `threads` host threads (0: all
 * cores), without FMA contraction, and loaded on the tape's device.  Values
 * cross a segment or stage boundary, and feed expectations and backward
 * partials, through the HBM tape (with recompute != 0, the backward kernel
 * first re-runs its segment's forward code, normals included, so only values
 * crossing a segment or stage boundary or feeding an expectation use the
 * tape; with recompute >= 2, the backward kernel does that in pieces of
 * `recompute` nodes, last piece first, each piece loading the values it needs
 * from earlier pieces, which the forward kernel then keeps on the tape: one
 * piece's values live in registers at a time); the rest of the evaluation (deterministic
 * nodes, expectations, fixed-order sums) is unchanged, so the results agree
 * with the interpreter's to the rounding of the reordered sums.  Later
 * mc_tape_value_and_grad calls run the compiled kernels.  Allocates a small
 * device table.  seconds_out: wall time of the compilation (or NULL);
 * hbm_bytes_out: HBM bytes per path of one compiled value and gradient (or
 * NULL).  MC_ERR_UNSUPPORTED if the run-time compiler fails (mc_tape_last_error
 * has the start of its log; the tape keeps interpreting). */
mc_status mc_tape_compile(mc_tape *t, int32_t seg_nodes, int32_t recompute, int32_t threads, double *seconds_out,
                          size_t *hbm_bytes_out);

/* Per-path value of node `node` on the last evaluated paths (FP64 device
 * [n_paths]); MC_ERR_INVALID_ARG for a deterministic node,
 * MC_ERR_UNSUPPORTED for a per-path node that is not kept on the tape (one
 * that only users fewer than 32 positions later in its stage read, and that
 * no backward partial needs; expectation arguments and arguments of
 * products, quotients, log, sqrt, relu and abs are always kept). */
mc_status mc_tape_path_values(mc_tape *t, int32_t node, double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MCTAPE_H */
