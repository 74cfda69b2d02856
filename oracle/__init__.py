"""FP64 CPU oracle for the KV-cache semantic operator (Sec. 5 of the Stretto paper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The CUDA product path never calls it, and this
package imports nothing from the CUDA path: the two share only the seeded input
generators in ``paper_2602_04430_b300.synth`` (which hold no arithmetic of the
method).

Modules
-------
``model``      Llama-style decoder primitives in float64 (RMSNorm, RoPE, GQA
               attention with an explicit visibility mask, SwiGLU FFN).
``operator``   The operator's steps in the paper's order: offline KV-cache
               creation (Sec. 5, "Offline: KV Cache Creation"), query-agnostic
               retention to a fraction r, online evaluation of the operator's
               prompt against the cache (Sec. 5, "Online: Query Execution"),
               the label logits and the accept / reject / unsure decision
               (Sec. 4.1, soft-threshold equation at temperature 0).
``fp8``        OCP FP8 E4M3 encode / decode and the per-block KV quantiser.
``proxy``      The learned proxy MLP: forward, backward, Adam, cascade merge
               (cascade recurrences of Sec. 4.1).

Parity status
-------------
Every function is pinned by tests in ``tests/test_oracle_*.py`` against closed
forms, library routines (torch fp64), brute force, or invariants the paper fixes
(a cached evaluation equals the from-scratch run, Sec. 5).  One part is
**parity unpinned**: the retention score ("EA-lite", ``operator.ea_scores``) is
this project's reading of the Expected Attention method the paper cites
without giving its formula; the score's own closed form (a Gaussian moment
generating function) is pinned, its fidelity to the cited method is not.
"""
