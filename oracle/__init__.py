"""FP64 CPU oracle of visibility stacking -- test infrastructure only.

Only tests/, the smoke check and the benchmark's CPU-baseline leg import this
package.  The GPU library never imports, links or runs it.
"""
