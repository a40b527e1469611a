// Internal types shared by the host code and the CUDA engine of the TTN
// trajectory simulator.  Not part of the C ABI.
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <vector>

#include "ttn.h"

namespace ttn {

// ---------------------------------------------------------------- circuit IR
// Op kinds of the syndrome-extraction circuit (Sec. III, Fig. 1).
enum OpKind { PREP_Z = 0, PREP_X = 1, CNOT = 2, MEAS_Z = 3, MEAS_X = 4, NOISE = 5 };

struct Op {
  int32_t kind, a, b, event, rec, layer;
};

// Triangular 6.6.6 color code (Sec. II.A, App. A.1).
struct Code {
  int d = 0, n = 0, P = 0;
  std::vector<std::array<int, 6>> dir;   // per face: neighbour qubit in lattice direction s, or -1
  std::vector<int> color;                // per face
  std::vector<std::vector<int>> support; // per face, sorted qubits
  std::vector<std::vector<int>> qplaqs;  // per qubit, sorted faces
};

Code build_code(int d);
std::vector<Op> build_ops(const Code& code, int rounds, int* n_layers, int* n_events,
                          int* n_locations);
std::vector<int> optimized_layout(const Code& code, const std::vector<Op>& ops, int n_qubits,
                                  int n_leaves);
// optimized_layout post-selected among `candidates` perturbed clusterings by
// the noise-free bond dimension; noise_free_bond_bits = log2 of that
// dimension for a layout (stabilizer tableau, host only).
std::vector<int> searched_layout(const Code& code, const std::vector<Op>& ops, int n_qubits,
                                 int n_leaves, int candidates);
int noise_free_bond_bits(const std::vector<Op>& ops, int n_qubits, int n_leaves,
                         const std::vector<int>& leaf_of_qubit);

// ---------------------------------------------------------------- device program
// One step of the per-trajectory program; every trajectory of a batch runs
// the same steps (the data-dependent part is only bond dimensions and values).
enum StepKind {
  S_MOVE = 0,        // a = v, b = w (neighbour), c = 1 if truncating (rank <= the bond's cap)
  S_THREAD_LEAF = 1, // a = node, b = leg (0 l / 1 r), c = factor set (0 control, 1 target)
  S_THREAD_NODE = 2, // a = node, b = leg towards the path child
  S_THREAD_LCA = 3,  // a = node (both child legs carry the MPO index)
  S_GATE_NODE = 4,   // a = node, b = 0 if control on leg l else 1
  S_LAYER1Q = 5,     // a = first entry, b = end entry of the 1q table, c = first group, d = end group
  S_MEASURE = 6,     // a = qubit, b = event, c = record bit, d = 1 for X basis
  S_AD = 7           // a = qubit, b = event
};

struct Step {
  int32_t kind, a, b, c, d, e;
};

// Fused single-qubit operations of one layer, grouped by the level-1 node
// that holds the qubit (both legs of one node are applied by one thread).
enum Op1Kind { O1_RESET_Z = 0, O1_RESET_X = 1, O1_SRX = 2, O1_PTA = 3 };

struct Op1 {
  int32_t leg, kind, qubit, event;
};

struct Group1 {
  int32_t node, begin, end, pad;
};

struct Program {
  std::vector<Step> steps;
  std::vector<Op1> op1;
  std::vector<Group1> groups;
  std::vector<int> stop_step_of_layer;  // index of the first step after layer L
};

// ---------------------------------------------------------------- decoder tables
// Concatenated MWPM decoder (App. A.2); see decoder.cu for the definition.
struct DecoderTables {
  int T = 0, P = 0, B = 0, n = 0;   // layers, faces, boundary node id, data qubits
  int n_nodes = 0;                  // B + 1
  std::vector<int32_t> color;       // [P]
  // stage 1, per colour c: all-pairs unit distances over node ids (-1: none)
  std::vector<int32_t> dist1;       // [3][n_nodes][n_nodes]
  std::vector<int32_t> adj1_off;    // [3][n_nodes + 1]
  std::vector<int32_t> adj1;        // neighbour lists, ascending
  std::vector<int32_t> adj1_base;   // [3] offset of colour c in adj1
  // per colour: the qubit sets of stage-1 space-edge classes ("non-c face sets")
  std::vector<int32_t> cls_off;     // [3][n_cls_max + 1] (prefix into cls_q)
  std::vector<int32_t> cls_q;       // qubits of each class, ascending
  std::vector<int32_t> cls_f;       // [3][n_cls_max][2] faces (-1 = boundary / none)
  std::vector<int32_t> n_cls;       // [3]
  int n_cls_max = 0;
  std::vector<int32_t> cface;       // [3][n] c-face of each qubit, -1 if none
  std::vector<int32_t> support_off; // [P + 1]
  std::vector<int32_t> support;     // face supports
};

DecoderTables build_decoder_tables(const Code& code, int rounds);

// All decoder tables packed into one int32 array (offsets in `off`), built
// once per circuit (host memory) so that the allocation-free decoder entry
// point only copies it into its static device table.
struct DecoderBlob {
  std::vector<int32_t> data;
  int32_t off[16] = {0};
};
DecoderBlob build_decoder_blob(const DecoderTables& t);

// ---------------------------------------------------------------- circuit handle
}  // namespace ttn

struct ttn_circuit {
  int d = 0, C = 0, n = 0, P = 0, N = 0, D = 0, L = 0;
  int n_layers = 0, n_events = 0, n_locations = 0, n_rec = 0;
  ttn::Code code;
  std::vector<ttn::Op> ops;
  std::vector<int> leaf_of_qubit;
  ttn::DecoderTables dec;
  // packed decoder tables, built by the first ttn_decode_noalloc call
  mutable ttn::DecoderBlob dec_blob;
  mutable bool dec_blob_ready = false;
};

namespace ttn {
Program compile_program(const ttn_circuit& c, int noise, int last_layer);

void set_error(const std::string& msg);
}  // namespace ttn
