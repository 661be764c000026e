"""Parquet enum values and Thrift field ids used by the oracle (test
infrastructure only).  Values follow the public parquet.thrift definition of
FileMetaData, RowGroup, ColumnChunk, ColumnMetaData, PageHeader and
OffsetIndex, the metadata of the hierarchy the paper's Section 2 describes."""

# Physical types
TYPE_ID = {"BOOLEAN": 0, "INT32": 1, "INT64": 2, "INT96": 3, "FLOAT": 4, "DOUBLE": 5,
           "BYTE_ARRAY": 6, "FIXED_LEN_BYTE_ARRAY": 7}
TYPE_NAME = {v: k for k, v in TYPE_ID.items()}

# Encodings
PLAIN, PLAIN_DICTIONARY, RLE, BIT_PACKED, DELTA_BINARY_PACKED = 0, 2, 3, 4, 5
DELTA_LENGTH_BYTE_ARRAY, DELTA_BYTE_ARRAY, RLE_DICTIONARY, BYTE_STREAM_SPLIT = 6, 7, 8, 9
ENCODING_ID = {"PLAIN": PLAIN, "RLE_DICTIONARY": RLE_DICTIONARY,
               "DELTA_BINARY_PACKED": DELTA_BINARY_PACKED,
               "DELTA_LENGTH_BYTE_ARRAY": DELTA_LENGTH_BYTE_ARRAY,
               "DELTA_BYTE_ARRAY": DELTA_BYTE_ARRAY, "BYTE_STREAM_SPLIT": BYTE_STREAM_SPLIT}

# Codecs
UNCOMPRESSED, SNAPPY, ZSTD = 0, 1, 6
CODEC_ID = {"UNCOMPRESSED": UNCOMPRESSED, "SNAPPY": SNAPPY, "ZSTD": ZSTD}

# Page types
DATA_PAGE, INDEX_PAGE, DICTIONARY_PAGE, DATA_PAGE_V2 = 0, 1, 2, 3

# Repetition
REQUIRED, OPTIONAL, REPEATED = 0, 1, 2
